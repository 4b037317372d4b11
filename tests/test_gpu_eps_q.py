"""eps_M at a finite momentum transfer on the molecular-crystal-like workload:
the mixed path (BF16x6 Hermitian plan, then the FP64 reduction, eigensolve and
spectrum) against the plain FP64 GPU path (FP64 build, the same FP64 steps),
paper Eqs. chir, osci and epsmtensor.  The reduced c5 shape (Nk = 8, 20 x 20
bands, NG = 500: N = 3,200) at Q index 3 (|Q| = 0.3 / bohr), inputs drawn on
the GPU.  Bars: every exciton energy within 1 meV, Im eps_M within 1e-3
relative at its peaks, A and B within 1e-6 relative Frobenius."""
import numpy as np
import pytest

import bse_inputs as bi

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
    assert m.mixed_available()
    return m


def _peaks(y, frac=0.1):
    return [i for i in range(1, len(y) - 1)
            if y[i] > y[i - 1] and y[i] >= y[i + 1] and y[i] > frac * y.max()]


@pytest.mark.parametrize("q_index", [3])
def test_eps_mixed_vs_fp64_at_finite_q(bse, q_index):
    import torch
    p = bi.make_problem_torch("c5s", q_index=q_index)
    assert float(np.linalg.norm(p["q_vec"])) > 0
    n = p["nk"] * p["nv"] * p["nc"]
    d = bse.upload_problem(p)
    A64, B64 = torch.empty_like(d["A"]), torch.empty_like(d["B"])
    om = torch.as_tensor(p["omega"]).cuda()
    rho = p["rho"] if torch.is_tensor(p["rho"]) else torch.as_tensor(p["rho"]).cuda()
    vc = p["nk"] * p["omega_cell"]
    bse.bse_build_kernel([bse.make_problem_struct(dict(d, A=A64, B=B64))], bse.BSE_PREC_FP64)
    plan = bse.Plan([bse.make_problem_struct(d)], precision=bse.BSE_PREC_BF16X6, hermitian=True)
    plan.execute()
    plan.status()
    plan.close()
    torch.cuda.synchronize()
    for X, X64 in ((d["A"], A64), (d["B"], B64)):
        assert ((X - X64).norm() / X64.norm()).item() < 1e-6
    out = []
    S = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    L = torch.empty_like(S)
    for A, B in ((A64, B64), (d["A"], d["B"])):
        E = torch.empty(n, dtype=torch.float64, device="cuda")
        osc = torch.empty_like(E)
        eps = torch.empty(len(p["omega"]), dtype=torch.complex128, device="cuda")
        bse.bse_reduce(n, A, B, S, L)
        bse.bse_spectrum(n, S, L, rho, p["c_q"], vc, om, p["delta"], E, osc, eps)
        torch.cuda.synchronize()
        out.append((E.cpu().numpy(), eps.cpu().numpy()))
    (e64, eps64), (emx, epsmx) = out
    assert np.abs(emx - e64).max() < 1e-3                       # 1 meV
    pk = _peaks(eps64.imag)
    assert len(pk) > 0
    rel = np.abs(epsmx.imag[pk] - eps64.imag[pk]) / np.abs(eps64.imag[pk])
    assert rel.max() < 1e-3
    print(f"\n[c5s Q index {q_index}: max dE {np.abs(emx - e64).max() * 1e3:.4f} meV, "
          f"{len(pk)} peaks, max rel d Im eps {rel.max():.2e}]", end="")
