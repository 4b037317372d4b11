"""Failure detection on the GPU without a fault: a bounded device wait made
to run out (a clock budget far below the time a tile's first operand copy
takes) ends the launch with a timeout status that bse_plan_status reports,
the context stays usable and the next execute is correct; the status word
keeps a timeout from an earlier execute until it is read; non-finite input
values are refused before any build (GPU)."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bse():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_05575_gb300 import build
    build.build()
    import paper_1904_05575_gb300 as m
    m.load()
    return m


def _rel(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


# the tensor-core stage 2 (pair blocks 64 x 64) and the fused direct term
CASES = [(bi.BSEConfig("f-tc", grid=2, nv=8, nc=8, ng=59, w_scale=0.05), {}),
         (bi.BSEConfig("f-fused", grid=2, nv=4, nc=4, ng=59, w_scale=0.1), {})]


@pytest.mark.parametrize("cfg,kw", CASES, ids=["tc-stage2", "fused"])
def test_wait_budget_expires_then_recovers(bse, cfg, kw):
    import torch
    p = bi.make_problem(cfg)
    A_ref, B_ref = O.build_A_B(p)
    d = bse.upload_problem(p)
    st = bse.make_problem_struct(d)
    plan = bse.Plan([st], precision=bse.BSE_PREC_BF16X6, **kw)
    # 1e-7 s is about 200 clock cycles: the first wait for an operand copy
    # (hundreds of nanoseconds at least) runs out in every CTA
    plan.set_wait_limit(1e-7)
    plan.execute()
    with pytest.raises(bse.BSEError) as err:
        plan.status()
    assert err.value.status == bse.BSE_ERR_TIMEOUT
    # the kernels returned and the context is usable: the default budget again
    plan.set_wait_limit(2.0)
    plan.execute()
    plan.status()
    torch.cuda.synchronize()
    n = p["nk"] * p["nv"] * p["nc"]
    assert _rel(bse.matrix_to_numpy(d["A"], n), A_ref) < 1e-6
    assert _rel(bse.matrix_to_numpy(d["B"], n), B_ref) < 1e-6
    plan.close()


def test_timeout_survives_later_execute_until_read(bse):
    """A timeout in the first of two executes (as when a captured graph is
    replayed several times before one status call) is still reported."""
    p = bi.make_problem(CASES[0][0])
    d = bse.upload_problem(p)
    plan = bse.Plan([bse.make_problem_struct(d)], precision=bse.BSE_PREC_BF16X6)
    plan.set_wait_limit(1e-7)
    plan.execute()
    plan.set_wait_limit(2.0)
    plan.execute()
    with pytest.raises(bse.BSEError) as err:
        plan.status()
    assert err.value.status == bse.BSE_ERR_TIMEOUT
    plan.status()            # read once: cleared
    plan.close()


@pytest.mark.parametrize("name", ["m_cc", "n_vc", "w", "e_v"])
def test_non_finite_input_refused(bse, name):
    import torch
    p = bi.make_problem(CASES[1][0])
    d = bse.upload_problem(p)
    d["A"].fill_(3.0)
    flat = d[name].view(-1)
    flat[flat.numel() // 2] = float("nan") if name != "e_v" else float("inf")
    st = bse.make_problem_struct(d)
    for prec in (bse.BSE_PREC_FP64, bse.BSE_PREC_BF16X6):
        with pytest.raises(bse.BSEError) as err:
            bse.bse_build_kernel([st], prec)
        assert err.value.status == bse.BSE_ERR_ARG and name in str(err.value)
    with pytest.raises(bse.BSEError) as err:
        bse.Plan([st], precision=bse.BSE_PREC_BF16X6)
    assert err.value.status == bse.BSE_ERR_ARG
    torch.cuda.synchronize()
    assert bool((d["A"] == 3.0).all()), "outputs untouched when the arguments are refused"
