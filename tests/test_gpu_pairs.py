"""Pair matrix elements from plane-wave coefficients on the GPU
(bse_pair_elements) against the oracle (oracle/pair_oracle.py), element by
element in FP64, whole and as k-row slabs; and the chain coefficients ->
pair elements -> Hamiltonian against the oracle's chain (GPU)."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O
from oracle import pair_oracle as PO

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


def _gpu(bse, n, cv, cc, basis, gout, kb=0, kn=0):
    import torch
    nk, nv, npw = cv.shape
    nc, ng = cc.shape[1], len(gout)
    rows = kn if kn else nk
    dev = lambda x: torch.as_tensor(x).cuda()
    out = {"m_x": torch.full((nk, nv, nc, ng), 9.0, dtype=torch.complex128, device="cuda"),
           "m_vv": torch.full((rows, nk, nv, nv, ng), 9.0, dtype=torch.complex128, device="cuda"),
           "m_cc": torch.full((rows, nk, nc, nc, ng), 9.0, dtype=torch.complex128, device="cuda"),
           "n_vc": torch.full((nk, nk, nv, nc, ng), 9.0, dtype=torch.complex128, device="cuda")}
    bse.bse_pair_elements(n, dev(cv), dev(cc), basis, gout, k_begin=kb, k_count=kn, **out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("n,nv,nc,npw,ng", [(2, 2, 3, 27, 15), (3, 2, 2, 15, 9), (1, 1, 1, 9, 1)],
                         ids=str)
def test_pair_elements_match_oracle(bse, n, nv, nc, npw, ng):
    cv, cc, basis = bi.wavefunction_coefficients(n, nv, nc, npw, seed=5)
    gout = bi.reciprocal_coords(ng)
    ref = PO.pair_elements(cv, cc, basis, gout, bi.k_grid(n), n)
    got = _gpu(bse, n, cv, cc, basis, gout)
    for name in ("m_x", "m_vv", "m_cc", "n_vc"):
        assert np.abs(got[name] - ref[name]).max() <= 1e-13 * max(np.abs(ref[name]).max(), 1.0), name


def test_pair_elements_slab_and_partial_outputs(bse):
    import torch
    n, nv, nc, npw, ng = 2, 2, 3, 27, 15
    cv, cc, basis = bi.wavefunction_coefficients(n, nv, nc, npw, seed=6)
    gout = bi.reciprocal_coords(ng)
    ref = PO.pair_elements(cv, cc, basis, gout, bi.k_grid(n), n, k_rows=range(4, 7))
    got = _gpu(bse, n, cv, cc, basis, gout, kb=4, kn=3)
    assert np.abs(got["m_vv"] - ref["m_vv"]).max() < 1e-13
    assert np.abs(got["m_cc"] - ref["m_cc"]).max() < 1e-13
    # one output only; the others stay untouched
    m_cc = torch.zeros((8, 8, nc, nc, ng), dtype=torch.complex128, device="cuda")
    bse.bse_pair_elements(n, torch.as_tensor(cv).cuda(), torch.as_tensor(cc).cuda(), basis, gout,
                          m_cc=m_cc)
    full = PO.pair_elements(cv, cc, basis, gout, bi.k_grid(n), n)
    assert np.abs(m_cc.cpu().numpy() - full["m_cc"]).max() < 1e-13
    with pytest.raises(bse.BSEError):
        bse.bse_pair_elements(n, torch.as_tensor(cv).cuda(), torch.as_tensor(cc).cuda(), basis, gout)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (2, 1e-6)], ids=["fp64", "bf16x6"])
def test_hamiltonian_from_coefficients(bse, prec, tol):
    """Coefficients -> pair elements (GPU) -> A, B (GPU) against coefficients ->
    pair elements (oracle) -> A, B (oracle); W, energies, maps and v from the
    input recipe of the same shape."""
    import torch
    n, nv, nc, npw, ng = 2, 2, 2, 27, 15
    cfg = bi.BSEConfig("coef", grid=n, nv=nv, nc=nc, ng=ng, w_scale=0.25)
    p = bi.make_problem(cfg, seed=9)
    cv, cc, basis = bi.wavefunction_coefficients(n, nv, nc, npw, seed=9)
    gout = bi.reciprocal_coords(ng)
    p.update(PO.pair_elements(cv, cc, basis, gout, bi.k_grid(n), n))
    A_ref, B_ref = O.build_A_B(p)
    d = bse.upload_problem(p)
    for name in ("m_x", "m_vv", "m_cc", "n_vc"):
        d[name].fill_(0.0)
    bse.bse_pair_elements(n, torch.as_tensor(cv).cuda(), torch.as_tensor(cc).cuda(), basis, gout,
                          m_x=d["m_x"], m_vv=d["m_vv"], m_cc=d["m_cc"], n_vc=d["n_vc"])
    bse.bse_build_kernel([bse.make_problem_struct(d)], prec)
    torch.cuda.synchronize()
    N = p["nk"] * nv * nc
    A, B = bse.matrix_to_numpy(d["A"], N), bse.matrix_to_numpy(d["B"], N)
    assert np.linalg.norm(A - A_ref) / np.linalg.norm(A_ref) < tol
    assert np.linalg.norm(B - B_ref) / np.linalg.norm(B_ref) < tol
