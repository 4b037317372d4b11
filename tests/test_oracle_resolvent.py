"""The resolvent form of the spectrum (CPU): the exciton sum of Eqs. chir and
osci, written with 1/(w - E + i d) - 1/(w + E + i d) = 2E/((w + i d)^2 - E^2),
equals (2 / V_c) conj(rho)^H ((w + i d)^2 - K)^-1 (A-B) conj(rho) with
K = (A-B)(A+B).  This is the reading bse_spectrum_lanczos evaluates (by a
Lanczos recursion); here it is checked against the oracle's spectrum from
the eigenpairs, by dense solves, and against mistakes in the reading."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O

HA = 27.211386245988


def _resolvent_eps(A, B, p, rho):
    n = A.shape[0]
    K = (A - B) @ (A + B)
    rb = np.conj(rho)
    vc = p["nk"] * p["omega_cell"]
    z2 = (p["omega"] + 1j * p["delta"]) ** 2
    Q = np.array([np.vdot(rb, np.linalg.solve(z * np.eye(n) - K, (A - B) @ rb)) for z in z2])
    return 1.0 - p["c_q"] * HA * (2.0 / vc) * Q


FINITE_Q = bi.BSEConfig("finite-q", grid=2, nv=2, nc=3, ng=27, q_abs=(0.4,), w_scale=0.2)


@pytest.mark.parametrize("cfg", ["c1", FINITE_Q], ids=["c1", "finite-q"])
def test_resolvent_equals_eigen_sum(cfg):
    p = bi.make_problem(cfg)
    A, B = O.build_A_B(p)
    eps_ref = O.spectrum(A, B, p)[2]
    eps = _resolvent_eps(A, B, p, p["rho"])
    assert np.abs(eps - eps_ref).max() < 1e-10 * np.abs(eps_ref).max()


def test_resolvent_reading_mutants():
    # the conjugate on rho, the factor (A-B) and the square of the frequency are
    # each needed: dropping any of them changes the spectrum
    p = bi.make_problem("c1")
    A, B = O.build_A_B(p)
    eps_ref = O.spectrum(A, B, p)[2]
    n = A.shape[0]
    vc = p["nk"] * p["omega_cell"]
    z = p["omega"] + 1j * p["delta"]
    K = (A - B) @ (A + B)
    scale = np.abs(eps_ref).max()

    def eps_of(q):
        return 1.0 - p["c_q"] * HA * (2.0 / vc) * q

    rho = p["rho"]
    no_conj = np.array([np.vdot(rho, np.linalg.solve(zz ** 2 * np.eye(n) - K, (A - B) @ rho))
                        for zz in z])
    no_amb = np.array([np.vdot(np.conj(rho), np.linalg.solve(zz ** 2 * np.eye(n) - K, np.conj(rho)))
                       for zz in z])
    linear = np.array([np.vdot(np.conj(rho), np.linalg.solve(zz * np.eye(n) - K, (A - B) @ np.conj(rho)))
                       for zz in z])
    for q in (no_conj, no_amb, linear):
        assert np.abs(eps_of(q) - eps_ref).max() > 1e-3 * scale
