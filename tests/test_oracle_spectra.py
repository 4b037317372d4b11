"""Pins of the oracle's Cartesian dielectric tensor, loss function and
dynamical structure factor (Eqs. tlambdai, epsmij, Lofeps and the S(Q, w)
definition), independent of their formulas:
  * contracting the tensor with a real unit vector q reproduces the scalar
    spectrum (itself pinned) for rho = sum_i q_i D_i (Eq. epsmtensor);
  * a one-transition problem worked by hand fixes the orientation t*_i t_j;
  * rotating the three directions rotates the tensor;
  * the loss is Im eps / |eps|^2, non-negative where Im eps >= 0, and
    S(Q, w) = (v_inv / pi) L."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O


def _three_directions(p, seed=3):
    """D [n, 3]: rho (= M_x at G = 0) and two seeded complex directions."""
    n = p["nk"] * p["nv"] * p["nc"]
    d = bi.directions(n, 2, seed=seed) * np.linalg.norm(p["rho"])
    return np.column_stack([p["rho"], d[:, 0], d[:, 1]])


@pytest.fixture(scope="module")
def c1():
    p = bi.make_problem("c1")
    A, B = O.build_A_B(p)
    e, xpy = O.solve_full(A, B)
    return p, e, xpy


def test_contraction_gives_the_scalar_spectrum(c1):
    p, e, xpy = c1
    vc = p["nk"] * p["omega_cell"]
    D = _three_directions(p)
    t = O.transition_coefficients(xpy, D, vc)
    eps3 = O.eps_tensor(e, t, p["omega"], p["delta"], p["c_q"])
    rng = np.random.default_rng(5)
    for _ in range(3):
        q = rng.standard_normal(3)
        q /= np.linalg.norm(q)
        scalar = O.eps_M(e, O.oscillator_strengths(xpy, D @ q, vc), p["omega"], p["delta"], p["c_q"])
        contracted = np.einsum("i,wij,j->w", q, eps3, q)
        assert np.abs(contracted - scalar).max() < 1e-12 * np.abs(scalar).max()
    for i in range(3):   # diagonal elements: the scalar spectrum of each direction
        scalar = O.eps_M(e, O.oscillator_strengths(xpy, D[:, i], vc), p["omega"], p["delta"], p["c_q"])
        assert np.abs(eps3[:, i, i] - scalar).max() < 1e-12 * np.abs(scalar).max()


def test_one_transition_by_hand():
    # N = 1: A = [a], B = [b]; E = sqrt((a - b)(a + b)), X - Y = (a + b)(X + Y)/E
    # and (X+Y)^* (X-Y) = 1 give |X+Y|^2 = E / (a + b); Eq. tlambdai then gives
    # t*_i t_j = |X+Y|^2 D_i conj(D_j) / V_c
    a, b, vc, c_q, delta = 3.0, 0.4, 2.5, 4 * np.pi, 0.05
    E = np.sqrt((a - b) * (a + b))
    xpy = np.array([[np.sqrt(E / (a + b)) * np.exp(0.3j)]])     # any phase
    D = np.array([[1.0 + 0.5j, 2.0j, -0.25]])
    t = O.transition_coefficients(xpy, D, vc)
    w = np.array([1.0, E, 5.0])
    eps3 = O.eps_tensor(np.array([E]), t, w, delta, c_q)
    res = 1 / (w - E + 1j * delta) + 1 / (-w - E - 1j * delta)
    coef = (E / (a + b)) * np.outer(D[0], np.conj(D[0])) / vc
    ref = np.eye(3)[None] - c_q * O.HARTREE_EV * coef[None] * res[:, None, None]
    assert np.abs(eps3 - ref).max() < 1e-13 * np.abs(ref).max()
    assert abs(eps3[1, 0, 1] - eps3[1, 1, 0]) > 1e-3       # not symmetric: orientation matters


def test_rotation_covariance(c1):
    p, e, xpy = c1
    vc = p["nk"] * p["omega_cell"]
    D = _three_directions(p)
    R, _ = np.linalg.qr(np.random.default_rng(7).standard_normal((3, 3)))
    eps3 = O.eps_tensor(e, O.transition_coefficients(xpy, D, vc), p["omega"], p["delta"], p["c_q"])
    epsR = O.eps_tensor(e, O.transition_coefficients(xpy, D @ R.T, vc), p["omega"], p["delta"], p["c_q"])
    ref = np.einsum("ai,wij,bj->wab", R, eps3, R)
    assert np.abs(epsR - ref).max() < 1e-12 * np.abs(ref).max()


def test_loss_and_structure_factor(c1):
    p, e, xpy = c1
    vc = p["nk"] * p["omega_cell"]
    eps = O.eps_M(e, O.oscillator_strengths(xpy, p["rho"], vc), p["omega"], p["delta"], p["c_q"])
    L = O.loss_function(eps)
    assert np.allclose(L, eps.imag / np.abs(eps) ** 2, rtol=1e-12, atol=0)
    pos = p["omega"] > 0
    assert (eps.imag[pos] >= 0).all() and (L[pos] >= 0).all()
    v_inv = 0.37 ** 2 / (4 * np.pi)
    assert np.allclose(O.structure_factor(eps, v_inv), v_inv / np.pi * L, rtol=1e-13, atol=0)
