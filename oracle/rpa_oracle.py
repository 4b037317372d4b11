"""Plain FP64 CPU oracle for the RPA screening that produces W (groundwork for
computing W on the GPU instead of taking it as an input).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only tests/ use it.  It shares no code with the CUDA
path.

Restates Sec. 2 of Vorwerk, Aurich, Cocchi, Draxl (arXiv:1904.05575): the
static screened interaction w_GG'(q) = v_G(q) eps^-1_GG'(q, omega = 0)
(Eq. wggq) with the dielectric matrix in the random-phase approximation (the
unnumbered equation after Eq. wggq).

Readings taken here (listed in the design notes):
  * An insulator at zero temperature: occupied = valence, unoccupied =
    conduction.  The sum over (i, j) has the pairs (v at k, c at k+q) and
    their reverses (c at k, v at k+q); at omega = 0 with time-reversal symmetry
    the two give the same contribution, so the sum is twice the (v, c) part.
  * Energies in eV and v in Hartree atomic units: 1/V_c times the 1/(energy)
    of the sum becomes kappa = Ha / (Nk Omega) over energies in eV, the same
    prefactor as in the Hamiltonian.
  * The conjugate is on the G factor, as printed: [M^G_ij]* M^G'_ij.

Parity status: pinned in tests/test_oracle_rpa.py by the no-transition limit,
a one-transition / one-plane-wave case and a two-plane-wave case worked by
hand, the Sherman-Morrison closed form for one transition, and the identity
w = (v^-1 + 2 kappa X)^-1 that makes w Hermitian with 0 < w <= v; seven
planted mistakes (factor, sign, conjugate and index placement, kappa) are
each caught by one of them.
"""
from __future__ import annotations

import numpy as np

from .bse_oracle import kappa


def rpa_sum(e_v: np.ndarray, e_c_kq: np.ndarray, m: np.ndarray) -> np.ndarray:
    """X_GG' = sum_{k v c} conj(M_vc,k(G)) M_vc,k(G') / (e_c(k+q) - e_v(k)).

    e_v [nk, nv] at k, e_c_kq [nk, nc] at k + q (eV), m [nk, nv, nc, ng]
    the pair elements M_vc(k, q)(G).  Returns [ng, ng] (eV^-1)."""
    nk, nv, nc, ng = m.shape
    x = np.zeros((ng, ng), np.complex128)
    for k in range(nk):
        for v in range(nv):
            for c in range(nc):
                de = e_c_kq[k, c] - e_v[k, v]
                x += np.outer(np.conj(m[k, v, c]), m[k, v, c]) / de
    return x


def rpa_epsilon(e_v: np.ndarray, e_c_kq: np.ndarray, m: np.ndarray, v_g: np.ndarray,
                omega_cell: float) -> np.ndarray:
    """eps^RPA_GG'(q, 0) = delta_GG' + 2 kappa v_G'(q) X_GG' (the RPA equation
    of Sec. 2 at omega = 0 for an insulator; the (f_j - f_i) / (e_j - e_i)
    factors are -1 / (e_c - e_v) for both orderings of each pair)."""
    nk = m.shape[0]
    x = rpa_sum(e_v, e_c_kq, m)
    return np.eye(len(v_g), dtype=np.complex128) + 2.0 * kappa(nk, omega_cell) * x * v_g[None, :]


def screened_w(eps: np.ndarray, v_g: np.ndarray) -> np.ndarray:
    """w_GG'(q) = v_G(q) eps^-1_GG'(q, 0) (Eq. wggq)."""
    return v_g[:, None] * np.linalg.inv(eps)
