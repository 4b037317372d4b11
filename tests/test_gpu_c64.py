"""Complex64 inputs (bse_problem.in_dtype = BSE_C64): the split-precision
build reads m_x, m_vv, m_cc, n_vc and w as complex64.  Every split rounds its
complex128 inputs to FP32 first, so the build from complex64 inputs equals,
bit for bit, the build from the same values stored as complex128, and both
match the oracle on those values (1e-6).  The paths that read complex128
refuse complex64."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O

pytestmark = pytest.mark.gpu

KEYS = ("m_x", "m_vv", "m_cc", "n_vc", "w")


@pytest.fixture(scope="module")
def bse():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_05575_gb300 import build
    build.build()
    import paper_1904_05575_gb300 as m
    m.load()
    assert m.mixed_available()
    return m


def _rounded(p):
    """The problem with its complex inputs rounded to complex64 and widened back."""
    q = dict(p)
    for k in KEYS:
        q[k] = np.asarray(p[k]).astype(np.complex64).astype(np.complex128)
    return q


def _rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


# pair blocks of >= 64 rows on both sides: every direct term on the tensor cores
@pytest.mark.parametrize("nv,nc,ng,herm", [(8, 8, 59, False), (8, 8, 300, True), (8, 9, 59, True)],
                         ids=str)
def test_c64_build_matches_c128_and_oracle(bse, nv, nc, ng, herm):
    import torch
    cfg = bi.BSEConfig(f"c64-{nv}-{nc}-{ng}", grid=2, nv=nv, nc=nc, ng=ng, w_scale=0.05)
    p = _rounded(bi.make_problem(cfg))
    A_ref, B_ref = O.build_A_B(p)
    n = p["nk"] * p["nv"] * p["nc"]
    outs = []
    for ct in (torch.complex128, torch.complex64):
        d = bse.upload_problem(p, complex_dtype=ct)
        assert d["m_x"].dtype == ct
        st = bse.make_problem_struct(d)
        assert st.in_dtype == (bse.BSE_C64 if ct == torch.complex64 else bse.BSE_C128)
        plan = bse.Plan([st], precision=bse.BSE_PREC_BF16X6, hermitian=herm)
        plan.execute()
        plan.status()
        plan.close()
        torch.cuda.synchronize()
        outs.append((d["A"].clone(), d["B"].clone()))
    (a128, b128), (a64, b64) = outs
    assert torch.equal(a128, a64) and torch.equal(b128, b64)
    assert _rel(bse.matrix_to_numpy(a64, n), A_ref) < 1e-6
    assert _rel(bse.matrix_to_numpy(b64, n), B_ref) < 1e-6


def test_c64_through_build_kernel(bse):
    import torch
    cfg = bi.BSEConfig("c64-bk", grid=2, nv=8, nc=8, ng=59, w_scale=0.05)
    p = _rounded(bi.make_problem(cfg))
    A_ref, B_ref = O.build_A_B(p)
    n = p["nk"] * p["nv"] * p["nc"]
    d = bse.upload_problem(p, complex_dtype=torch.complex64)
    bse.bse_build_kernel([bse.make_problem_struct(d)], bse.BSE_PREC_BF16X6)
    torch.cuda.synchronize()
    assert _rel(bse.matrix_to_numpy(d["A"], n), A_ref) < 1e-6
    assert _rel(bse.matrix_to_numpy(d["B"], n), B_ref) < 1e-6


def test_c64_refusals(bse):
    import torch
    big = bse.upload_problem(_rounded(bi.make_problem(
        bi.BSEConfig("c64-r", grid=2, nv=8, nc=8, ng=59, w_scale=0.05))), complex_dtype=torch.complex64)
    st = bse.make_problem_struct(big)
    for call in (lambda: bse.bse_build_kernel([st], bse.BSE_PREC_FP64),
                 lambda: bse.bse_build_kernel_fp64_static(st),
                 lambda: bse.Plan([st], precision=bse.BSE_PREC_BF16X6, fp64_diagonal=True),
                 lambda: bse.Plan([st], precision=bse.BSE_PREC_BF16X6, tc_stage2=False)):
        with pytest.raises(bse.BSEError) as ei:
            call()
        assert ei.value.status == bse.BSE_ERR_UNSUPPORTED
    # small pair blocks need the CUDA-core stage 2 (or the fused term): refused
    small = bse.upload_problem(bi.make_problem("c1"), complex_dtype=torch.complex64)
    with pytest.raises(bse.BSEError) as ei:
        bse.bse_build_kernel([bse.make_problem_struct(small)], bse.BSE_PREC_BF16X6)
    assert ei.value.status == bse.BSE_ERR_UNSUPPORTED
    # a planted NaN in a complex64 input is found by the scan
    big["m_cc"].view(torch.float32).view(-1)[12345] = float("nan")
    with pytest.raises(bse.BSEError) as ei:
        bse.Plan([bse.make_problem_struct(big)], precision=bse.BSE_PREC_BF16X6)
    assert ei.value.status == bse.BSE_ERR_ARG and "m_cc" in str(ei.value)
