"""The exact FP64 diagonal after a split-precision build (BSE_PLAN_FP64_DIAGONAL):
A_aa and B_aa match the oracle's to 1e-12 relative on every stage-2 path, k-row
slabs and Hermitian plans, and every off-diagonal element is the one the plan
without the flag writes (GPU)."""
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


CASES = {
    "tc-stage2": bi.BSEConfig("d-tc", grid=2, nv=8, nc=8, ng=59, w_scale=0.05),
    "fused": bi.BSEConfig("d-fused", grid=2, nv=4, nc=4, ng=59, w_scale=0.1),
    "cuda-core": bi.BSEConfig("d-cc", grid=2, nv=3, nc=5, ng=59, w_scale=0.1),
    "core-like": bi.BSEConfig("d-core", grid=2, nv=2, nc=20, ng=59, w_scale=0.25,
                              e_v_range=(-400.5, -399.5), m_decay=0.05),
}


def _build(bse, p, **kw):
    import torch
    d = bse.upload_problem(p)
    plan = bse.Plan([bse.make_problem_struct(d)], precision=bse.BSE_PREC_BF16X6, **kw)
    plan.execute()
    plan.status()
    torch.cuda.synchronize()
    n = p["nk"] * p["nv"] * p["nc"]
    out = bse.matrix_to_numpy(d["A"], n), bse.matrix_to_numpy(d["B"], n)
    plan.close()
    return out


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("hermitian", [False, True], ids=["all-blocks", "hermitian"])
def test_fp64_diagonal_matches_oracle(bse, name, hermitian):
    p = bi.make_problem(CASES[name])
    A_ref, B_ref = O.build_A_B(p)
    A, B = _build(bse, p, fp64_diagonal=True, hermitian=hermitian)
    for M, R in ((A, A_ref), (B, B_ref)):
        d, dr = np.diag(M), np.diag(R)
        assert np.abs(d.imag).max() == 0.0
        assert np.abs(d.real - dr.real).max() <= 1e-12 * np.abs(dr).max()
    # the split-precision diagonal alone is ~1e-7 off; the rest is the plain build
    A0, B0 = _build(bse, p, hermitian=hermitian)
    off = ~np.eye(A.shape[0], dtype=bool)
    assert np.array_equal(A[off], A0[off]) and np.array_equal(B[off], B0[off])


def test_fp64_diagonal_slab_rows(bse):
    import torch
    cfg = CASES["tc-stage2"]
    p = bi.make_problem(cfg)
    A_ref, B_ref = O.build_A_B(p)
    nk, nb = p["nk"], p["nv"] * p["nc"]
    d = bse.upload_problem(p)
    full_vv, full_cc = d["m_vv"], d["m_cc"]
    for kb in (0, 4):
        d["m_vv"], d["m_cc"] = full_vv[kb:kb + 4].contiguous(), full_cc[kb:kb + 4].contiguous()
        plan = bse.Plan([bse.make_problem_struct(d, k_begin=kb, k_count=4)],
                        precision=bse.BSE_PREC_BF16X6, fp64_diagonal=True)
        plan.execute()
        plan.status()
        plan.close()
    torch.cuda.synchronize()
    n = nk * nb
    A, B = bse.matrix_to_numpy(d["A"], n), bse.matrix_to_numpy(d["B"], n)
    assert np.abs(np.diag(A).real - np.diag(A_ref).real).max() <= 1e-12 * np.abs(np.diag(A_ref)).max()
    assert np.abs(np.diag(B).real - np.diag(B_ref).real).max() <= 1e-12 * np.abs(np.diag(B_ref)).max()
