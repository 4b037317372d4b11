"""eps_M by the Lanczos recursion on (A-B)(A+B) (bse_spectrum_lanczos) against
the oracle's spectrum from the eigenpairs (paper Eqs. chir, osci,
epsmtensor), and on the reduced molecular-crystal shape against the FP64
GPU path (reduction, eigensolve, spectrum); argument and breakdown cases."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O

pytestmark = pytest.mark.gpu

FINITE_Q = bi.BSEConfig("finite-q-lz", grid=2, nv=2, nc=3, ng=27, q_abs=(0.4,), w_scale=0.2)
RAGGED = bi.BSEConfig("ragged-lz", grid=3, nv=3, nc=5, ng=59, w_scale=0.1)   # N = 405


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


def _t(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def _gpu_matrix(M):
    return _t(np.ascontiguousarray(M.T))


@pytest.mark.parametrize("prec", [0, 2], ids=["fp64", "bf16x6"])
@pytest.mark.parametrize("cfg", ["c1", FINITE_Q, RAGGED, "c2"], ids=["c1", "finite-q", "ragged", "c2"])
def test_lanczos_matches_oracle_spectrum(bse, cfg, prec):
    """FP64 products: eps to 1e-7 of the oracle (1e-6 at the peaks); tensor-core
    products (BF16x6): to 1e-5 (1e-4 at the peaks)."""
    import torch
    p = bi.make_problem(cfg)
    A, B = O.build_A_B(p)
    n = A.shape[0]
    eps_ref = O.spectrum(A, B, p)[2]
    eps = torch.empty(len(p["omega"]), dtype=torch.complex128, device="cuda")
    steps = bse.bse_spectrum_lanczos(n, _gpu_matrix(A), _gpu_matrix(B), _t(p["rho"]), p["c_q"],
                                     p["nk"] * p["omega_cell"], _t(p["omega"]), p["delta"], eps,
                                     tol=1e-10, matvec_precision=prec)
    e = eps.cpu().numpy()
    scale = np.abs(eps_ref).max()
    bound, bound_pk = (1e-7, 1e-6) if prec == 0 else (1e-5, 1e-4)
    assert np.abs(e - eps_ref).max() < bound * scale
    y = eps_ref.imag
    pk = [i for i in range(1, len(y) - 1) if y[i] > y[i - 1] and y[i] >= y[i + 1] and y[i] > 0.1 * y.max()]
    assert len(pk) > 0
    assert (np.abs(e[pk] - eps_ref[pk]) / np.abs(eps_ref[pk])).max() < bound_pk
    print(f" [{steps} steps]", end="")


@pytest.mark.parametrize("prec", [0, 2], ids=["fp64", "bf16x6"])
def test_lanczos_matches_fp64_path_on_reduced_crystal(bse, prec):
    """The reduced molecular-crystal shape (N = 3,200, NG = 500) at a finite Q:
    the mixed build, then eps by the recursion, against the FP64 build, the
    reduction, the eigensolve and the spectrum; Im eps within 1e-3 at the peaks."""
    import torch
    p = bi.make_problem_torch("c5s", q_index=3)
    n = p["nk"] * p["nv"] * p["nc"]
    d = bse.upload_problem(p)
    A64, B64 = torch.empty_like(d["A"]), torch.empty_like(d["B"])
    bse.bse_build_kernel([bse.make_problem_struct(dict(d, A=A64, B=B64))], bse.BSE_PREC_FP64)
    plan = bse.Plan([bse.make_problem_struct(d)], precision=bse.BSE_PREC_BF16X6, hermitian=True)
    plan.execute()
    plan.status()
    plan.close()
    om = torch.as_tensor(p["omega"]).cuda()
    rho = p["rho"] if torch.is_tensor(p["rho"]) else _t(p["rho"])
    vc = p["nk"] * p["omega_cell"]
    S = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    L = torch.empty_like(S)
    E = torch.empty(n, dtype=torch.float64, device="cuda")
    osc = torch.empty_like(E)
    eps64 = torch.empty(len(p["omega"]), dtype=torch.complex128, device="cuda")
    bse.bse_reduce(n, A64, B64, S, L)
    bse.bse_spectrum(n, S, L, rho, p["c_q"], vc, om, p["delta"], E, osc, eps64)
    eps = torch.empty_like(eps64)
    steps = bse.bse_spectrum_lanczos(n, d["A"], d["B"], rho, p["c_q"], vc, om, p["delta"], eps,
                                     tol=1e-8, matvec_precision=prec)
    e, r = eps.cpu().numpy(), eps64.cpu().numpy()
    y = r.imag
    pk = [i for i in range(1, len(y) - 1) if y[i] > y[i - 1] and y[i] >= y[i + 1] and y[i] > 0.1 * y.max()]
    assert len(pk) > 0
    rel = np.abs(e.imag[pk] - y[pk]) / np.abs(y[pk])
    assert rel.max() < 1e-3
    print(f" [c5s: {steps} steps, max rel d Im eps at {len(pk)} peaks {rel.max():.1e}]", end="")


def test_lanczos_errors(bse):
    import torch
    p = bi.make_problem("c1")
    A, B = O.build_A_B(p)
    n = A.shape[0]
    om = _t(p["omega"])
    eps = torch.empty(len(p["omega"]), dtype=torch.complex128, device="cuda")
    vc = p["nk"] * p["omega_cell"]
    with pytest.raises(bse.BSEError) as ei:      # rho = 0
        bse.bse_spectrum_lanczos(n, _gpu_matrix(A), _gpu_matrix(B), _t(np.zeros(n, complex)),
                                 p["c_q"], vc, om, p["delta"], eps)
    assert ei.value.status == bse.BSE_ERR_ARG
    with pytest.raises(bse.BSEError) as ei:      # A - B negative definite
        bse.bse_spectrum_lanczos(n, _gpu_matrix(-np.eye(n, dtype=complex)), None, _t(p["rho"]),
                                 p["c_q"], vc, om, p["delta"], eps)
    assert ei.value.status == bse.BSE_ERR_NOT_PD
    with pytest.raises(bse.BSEError) as ei:      # too few steps allowed
        bse.bse_spectrum_lanczos(n, _gpu_matrix(A), _gpu_matrix(B), _t(p["rho"]), p["c_q"], vc,
                                 om, p["delta"], eps, tol=1e-14, max_steps=20)
    assert ei.value.status == bse.BSE_ERR_NO_CONV and ei.value.steps == 20
    assert np.isfinite(eps.cpu().numpy()).all()
    with pytest.raises(bse.BSEError):            # delta must be > 0
        bse.bse_spectrum_lanczos(n, _gpu_matrix(A), _gpu_matrix(B), _t(p["rho"]), p["c_q"], vc,
                                 om, 0.0, eps)
