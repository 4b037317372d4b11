"""Hermitian plans (BSE_PLAN_HERMITIAN): the direct terms built over the
blocks k <= k' only and the blocks k > k' completed from their mirrors
(A and B Hermitian, Eq. Hetr), against the oracle's full build and against
the plan that computes every block, on every stage-2 path (tensor-core pair
blocks, CUDA-core pair blocks, the fused direct term); the exchange written
over the blocks k <= k' and completed, with and without the flag (GPU)."""
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


def _build(bse, probs, prec, **kw):
    import torch
    ds = [bse.upload_problem(p) for p in probs]
    sts = [bse.make_problem_struct(d) for d in ds]
    plan = bse.Plan(sts, precision=prec, **kw)
    for _ in range(2):                 # a plan is reusable: the second execute starts from garbage
        for d in ds:
            d["A"].fill_(7.0)
            d["B"].fill_(-3.0)
        plan.execute()
        plan.status()
    torch.cuda.synchronize()
    out = []
    for p, d in zip(probs, ds):
        n = p["nk"] * p["nv"] * p["nc"]
        out.append((bse.matrix_to_numpy(d["A"], n), bse.matrix_to_numpy(d["B"], n)))
    plan.close()
    return out


def _blocks_mirror_exactly(M, nb):
    """Elements of blocks k > k' are exact conjugates of their mirrors."""
    n = M.shape[0]
    k = np.arange(n) // nb
    low = k[:, None] > k[None, :]
    return np.array_equal(M[low], M.T.conj()[low])


# pair blocks of 64 x 64 (Nv = Nc = 8): both stage-2 contractions on the tensor
# cores; Nv = 8, Nc = 9 puts the W^rr stage-1 side on (v, v'); NG = 300 cuts K
# into segments
TC_CASES = [bi.BSEConfig("h-tc-8-8", grid=2, nv=8, nc=8, ng=59, w_scale=0.05),
            bi.BSEConfig("h-tc-8-9", grid=2, nv=8, nc=9, ng=59, w_scale=0.05),
            bi.BSEConfig("h-tc-8-8-300", grid=2, nv=8, nc=8, ng=300, w_scale=0.05)]
# CUDA-core pair blocks (uneven windows, three Q in one plan) and the fused
# direct term (Nv = Nc in {2, 4})
MULTI = bi.BSEConfig("h-multi", grid=2, nv=4, nc=6, ng=59, q_abs=(0.1, 0.6, 1.1),
                     windows=((2, 2), (3, 5), (4, 6)), w_scale=0.1)
SQUARE = bi.BSEConfig("h-square", grid=2, nv=4, nc=4, ng=59, q_abs=(0.1, 0.6, 1.1),
                      windows=((2, 2), (4, 4), (2, 2)), w_scale=0.1)


@pytest.mark.parametrize("cfg", TC_CASES, ids=lambda c: c.name)
def test_hermitian_tensor_core_stage2(bse, cfg):
    p = bi.make_problem(cfg)
    A_ref, B_ref = O.build_A_B(p)
    (A, B), = _build(bse, [p], bse.BSE_PREC_BF16X6, hermitian=True)
    assert _rel(A, A_ref) < 1e-6 and _rel(B, B_ref) < 1e-6
    nb = p["nv"] * p["nc"]
    assert _blocks_mirror_exactly(A, nb) and _blocks_mirror_exactly(B, nb)
    (A2, B2), = _build(bse, [p], bse.BSE_PREC_BF16X6)
    assert _rel(A, A2) < 1e-6 and _rel(B, B2) < 1e-6


@pytest.mark.parametrize("cfg,fused", [(MULTI, False), (SQUARE, True)], ids=["cuda-core", "fused"])
def test_hermitian_small_blocks(bse, cfg, fused):
    probs = [bi.make_problem(cfg, q_index=q) for q in range(3)]
    refs = [O.build_A_B(p) for p in probs]
    outs = _build(bse, probs, bse.BSE_PREC_BF16X6, hermitian=True, fused=fused)
    for p, (A_ref, B_ref), (A, B) in zip(probs, refs, outs):
        assert _rel(A, A_ref) < 1e-6 and _rel(B, B_ref) < 1e-6
        nb = p["nv"] * p["nc"]
        assert _blocks_mirror_exactly(A, nb) and _blocks_mirror_exactly(B, nb)


def test_hermitian_tda_leaves_b(bse):
    import torch
    p = bi.make_problem(TC_CASES[0])
    A_ref, _ = O.build_A_B(p, coupling=False)
    d = bse.upload_problem(p)
    d["B"].fill_(5.0)
    st = bse.make_problem_struct(d, coupling=False)
    plan = bse.Plan([st], precision=bse.BSE_PREC_BF16X6, hermitian=True)
    plan.execute()
    plan.status()
    torch.cuda.synchronize()
    n = p["nk"] * p["nv"] * p["nc"]
    assert _rel(bse.matrix_to_numpy(d["A"], n), A_ref) < 1e-6
    assert bool((d["B"] == 5.0).all())
    plan.close()


# N = 3,072 on a 4x4x4 grid: enough exchange tiles (at least two per SM) that
# the exchange writes the blocks k <= k' only and the rest is completed, with
# and without the flag
UPPER = bi.BSEConfig("h-upper", grid=4, nv=4, nc=12, ng=59, w_scale=0.1)


@pytest.mark.parametrize("hermitian", [False, True], ids=["all-blocks", "hermitian"])
def test_exchange_upper_blocks_completed(bse, hermitian):
    p = bi.make_problem(UPPER)
    A_ref, B_ref = O.build_A_B(p)
    (A, B), = _build(bse, [p], bse.BSE_PREC_BF16X6, hermitian=hermitian)
    assert _rel(A, A_ref) < 1e-6 and _rel(B, B_ref) < 1e-6
    # the real-valued diagonal of A carries the transition energies
    e = O.transition_energies(p["e_v"], p["e_c"])
    assert np.abs(np.diag(A).imag).max() == 0.0
    assert np.allclose(np.diag(A).real, np.diag(A_ref).real, rtol=1e-6, atol=1e-6)
    nb = p["nv"] * p["nc"]
    if hermitian:
        assert _blocks_mirror_exactly(A, nb) and _blocks_mirror_exactly(B, nb)
    # the exchange alone (gamma_c = 0): V is Hermitian for any M_x
    import torch
    d = bse.upload_problem(p)
    st = bse.make_problem_struct(d, gamma_c=0.0)
    plan = bse.Plan([st], precision=bse.BSE_PREC_BF16X6, hermitian=hermitian)
    plan.execute()
    plan.status()
    torch.cuda.synchronize()
    Ax_ref, Bx_ref = O.build_A_B(p, gamma_c=0.0)
    n = p["nk"] * p["nv"] * p["nc"]
    Ax, Bx = bse.matrix_to_numpy(d["A"], n), bse.matrix_to_numpy(d["B"], n)
    assert _rel(Ax - np.diag(e), Ax_ref - np.diag(e)) < 1e-6 and _rel(Bx, Bx_ref) < 1e-6
    assert _blocks_mirror_exactly(Bx, nb)
    plan.close()


def test_hermitian_plan_rejects_slabs(bse):
    p = bi.make_problem(TC_CASES[0])
    d = bse.upload_problem(p)
    d["m_vv"], d["m_cc"] = d["m_vv"][:4].contiguous(), d["m_cc"][:4].contiguous()
    st = bse.make_problem_struct(d, k_begin=0, k_count=4)
    with pytest.raises(bse.BSEError) as err:
        bse.Plan([st], precision=bse.BSE_PREC_BF16X6, hermitian=True)
    assert err.value.status == bse.BSE_ERR_UNSUPPORTED
