"""Cartesian dielectric tensor, loss function and dynamical structure factor
on the GPU (Eqs. tlambdai, epsmij, Lofeps, S(Q, w)) against the oracle,
through the C ABI, on the FP64 build of c1 and c2 and at a finite Q."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O
from test_gpu_fp64 import gpu_build, problem

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


def _directions(p):
    n = p["nk"] * p["nv"] * p["nc"]
    d = bi.directions(n, 2, seed=3) * np.linalg.norm(p["rho"])
    return np.column_stack([p["rho"], d[:, 0], d[:, 1]])


@pytest.mark.parametrize("name,q", [("c1", 0), ("c2", 0), ("c1-finite-q", 0)])
def test_tensor_loss_structure_factor_match_oracle(bse, name, q):
    import torch
    if name == "c1-finite-q":
        p = bi.make_problem(bi.BSEConfig("c1q", grid=2, nv=2, nc=2, ng=59, q_abs=(0.35,),
                                         w_scale=0.25))
    else:
        p = problem(name)
    n = p["nk"] * p["nv"] * p["nc"]
    vc = p["nk"] * p["omega_cell"]
    A, B = O.build_A_B(p)
    e_ref, xpy = O.solve_full(A, B)
    D = _directions(p)
    eps3_ref = O.eps_tensor(e_ref, O.transition_coefficients(xpy, D, vc), p["omega"], p["delta"],
                            p["c_q"])
    d = gpu_build(bse, p)
    S = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    L = torch.empty_like(S)
    bse.bse_reduce(n, d["A"], d["B"], S, L)
    E = torch.empty(n, dtype=torch.float64, device="cuda")
    osc = torch.empty_like(E)
    om = torch.as_tensor(p["omega"]).cuda()
    eps = torch.empty(len(p["omega"]), dtype=torch.complex128, device="cuda")
    bse.bse_spectrum(n, S, L, torch.as_tensor(p["rho"]).cuda(), p["c_q"], vc, om, p["delta"],
                     E, osc, eps)
    eps3 = torch.empty((len(p["omega"]), 3, 3), dtype=torch.complex128, device="cuda")
    bse.bse_spectrum_tensor(n, S, L, torch.as_tensor(np.ascontiguousarray(D.T)).cuda(), p["c_q"],
                            vc, om, p["delta"], E, eps3)
    got = eps3.cpu().numpy()
    assert np.abs(got - eps3_ref).max() < 1e-9 * np.abs(eps3_ref).max()
    # rho is the first direction: the (0, 0) element is bse_spectrum's eps_M
    assert np.abs(got[:, 0, 0] - eps.cpu().numpy()).max() < 1e-12 * np.abs(got[:, 0, 0]).max()
    # loss function and S(Q, w) of the scalar eps_M
    v_inv = (np.linalg.norm(p["q_vec"]) ** 2 if np.linalg.norm(p["q_vec"]) > 0 else 1.0) / (4 * np.pi)
    loss = torch.empty(len(p["omega"]), dtype=torch.float64, device="cuda")
    sqw = torch.empty_like(loss)
    bse.bse_loss_function(eps, v_inv, loss, sqw)
    torch.cuda.synchronize()
    eps_np = eps.cpu().numpy()
    L_ref = O.loss_function(eps_np)
    assert np.abs(loss.cpu().numpy() - L_ref).max() < 1e-12 * np.abs(L_ref).max()
    S_ref = O.structure_factor(eps_np, v_inv)
    assert np.abs(sqw.cpu().numpy() - S_ref).max() < 1e-12 * np.abs(S_ref).max()
