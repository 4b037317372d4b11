"""Plain CPU oracle for the plane-wave pair matrix elements from wavefunction
coefficients (the matrix elements M and N of the LAPW section, interstitial
part: the whole element for wavefunctions expanded in plane waves only).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py use it.  It shares no code with the
CUDA path.

A Bloch function phi_{nk}(r) = sum_{G in S} C_{nk}(G) e^{i(k+G)r} (unit-norm
plane waves over the crystal volume) has, for q on the k grid and the
reciprocal-lattice vector s that brings k + q back to the grid point it
lands on,
  M(a, b; G, s) = <a| e^{-i(G+q)r} |b> = sum_{G1 in S} conj(a(G1)) b(G1 + G + s)
  N(a, b; G, s) = <a| e^{-i(G+q)r} |b^*> = sum_{G1 in S} conj(a(G1)) conj(b(-G1 - G - s))
with b(G) = 0 for G outside S (orthogonality of the plane waves: the
integral keeps the terms whose wave vectors cancel).  The BSE inputs follow
the conventions of the C ABI (include/bse.h), all at Q = 0:
  m_x[k][v][c](G)        = <c k| e^{-iGr} |v k>                               (Eq. vrrofM)
  m_vv[k][k'][v][v'](G)  = <v' k'| e^{-i(G+q)r} |v k>,  q = k - k' on the grid (Eq. wrrm)
  m_cc[k][k'][c][c'](G)  = <c' k'| e^{-i(G+q)r} |c k>
  n_vc[k][k'][v][c'](G)  = <v k| e^{-i(G+q)r} |(c' k')^*>, q = -k - k'         (Eq. wrabar)
Reciprocal vectors are integer coordinates in the reciprocal-lattice basis;
k points are integer coordinates in units of 1/n of it (an n^3 grid).
"""
from __future__ import annotations

from typing import Dict, Sequence, Tuple

import numpy as np


def _lookup(basis: np.ndarray):
    """Dictionary from an integer coordinate triple to its index in basis."""
    return {tuple(int(x) for x in g): i for i, g in enumerate(basis)}


def element_m(a: np.ndarray, b: np.ndarray, basis: np.ndarray, G: np.ndarray, s) -> complex:
    """M(a, b; G, s) = sum_{G1 in S} conj(a(G1)) b(G1 + G + s)."""
    idx = _lookup(basis)
    tot = 0.0 + 0.0j
    for i1, g1 in enumerate(basis):
        j = idx.get(tuple(int(x) for x in (g1 + G + s)))
        if j is not None:
            tot += np.conj(a[i1]) * b[j]
    return tot


def element_n(a: np.ndarray, b: np.ndarray, basis: np.ndarray, G: np.ndarray, s) -> complex:
    """N(a, b; G, s) = sum_{G1 in S} conj(a(G1)) conj(b(-G1 - G - s))."""
    idx = _lookup(basis)
    tot = 0.0 + 0.0j
    for i1, g1 in enumerate(basis):
        j = idx.get(tuple(int(x) for x in (-g1 - G - s)))
        if j is not None:
            tot += np.conj(a[i1]) * np.conj(b[j])
    return tot


def umklapp(kint: np.ndarray, n: int, k: int, kp: int, sign: int) -> Tuple[int, np.ndarray]:
    """Grid index of q and the reciprocal vector s (integer coordinates) with
    k' + q - k = n s for q = k - k' on the grid (sign = -1), or k + k' + q = n s
    for q = -k - k' (sign = +1); k, q in units of 1/n of the reciprocal basis."""
    if sign < 0:
        qi = kint[k] - kint[kp]
    else:
        qi = -kint[k] - kint[kp]
    qg = np.mod(qi, n)
    q_index = int((qg[0] * n + qg[1]) * n + qg[2])
    if sign < 0:
        s = (kint[kp] + qg - kint[k]) // n          # k' + q - k = n s: ket term G1 + G + s
        return q_index, s
    s = (kint[k] + kint[kp] + qg) // n              # k + k' + q = n s: ket term -G1 - G - s
    return q_index, s


def pair_elements(cv: np.ndarray, cc: np.ndarray, basis: np.ndarray, gout: np.ndarray,
                  kint: np.ndarray, n: int, k_rows: Sequence[int] | None = None) -> Dict:
    """m_x, m_vv, m_cc (rows k_rows), n_vc (whole) from coefficients
    cv [nk][nv][npw], cc [nk][nc][npw] over the basis [npw][3], at the output
    vectors gout [ng][3]; nested loops over the definitions above."""
    nk, nv, _ = cv.shape
    nc = cc.shape[1]
    ng = len(gout)
    k_rows = list(range(nk)) if k_rows is None else list(k_rows)
    zero = np.zeros(3, dtype=np.int64)
    m_x = np.empty((nk, nv, nc, ng), np.complex128)
    for k in range(nk):
        for v in range(nv):
            for c in range(nc):
                for g in range(ng):
                    m_x[k, v, c, g] = element_m(cc[k, c], cv[k, v], basis, gout[g], zero)
    m_vv = np.empty((len(k_rows), nk, nv, nv, ng), np.complex128)
    m_cc = np.empty((len(k_rows), nk, nc, nc, ng), np.complex128)
    for r, k in enumerate(k_rows):
        for kp in range(nk):
            _, s = umklapp(kint, n, k, kp, -1)
            for v in range(nv):
                for vp in range(nv):
                    for g in range(ng):
                        m_vv[r, kp, v, vp, g] = element_m(cv[kp, vp], cv[k, v], basis, gout[g], s)
            for c in range(nc):
                for cp in range(nc):
                    for g in range(ng):
                        m_cc[r, kp, c, cp, g] = element_m(cc[kp, cp], cc[k, c], basis, gout[g], s)
    n_vc = np.empty((nk, nk, nv, nc, ng), np.complex128)
    for k in range(nk):
        for kp in range(nk):
            _, s = umklapp(kint, n, k, kp, +1)
            for v in range(nv):
                for cp in range(nc):
                    for g in range(ng):
                        n_vc[k, kp, v, cp, g] = element_n(cv[k, v], cc[kp, cp], basis, gout[g], s)
    return dict(m_x=m_x, m_vv=m_vv, m_cc=m_cc, n_vc=n_vc)
