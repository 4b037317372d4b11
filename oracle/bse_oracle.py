"""Plain FP64 CPU oracle for the BSE Hamiltonian build, reduction and spectrum.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py use it.  It shares no code with the
CUDA path; both take their inputs from bse_inputs.

Every function restates one passage of Vorwerk, Aurich, Cocchi, Draxl,
"Bethe-Salpeter equation for absorption and scattering spectroscopy:
Implementation in the exciting code" (arXiv:1904.05575), cited by section and
equation label.  Loops run over the k / k' pairs the way the equations are
written; numpy einsum / matmul / eigh serve only as library steps.

Readings of the paper taken here (each listed in the design notes):
  * Coulomb potential v_G(Q) = 4 pi / |G+Q|^2 with the G = 0 term removed
    (Eq. vft prints |G+q| without the square; Eq. vbar_def removes the term).
  * One prefactor kappa = Ha / (Nk * Omega) = Ha / V_c multiplies V, W^rr and
    W^ra (Eq. vft carries 1/V_c, Eq. wrabar prints 1/V); energies are in eV.
  * B is Hermitian (Eq. Hetr in the time-reversal basis), so the brute-force
    form is Delta H = [[A, B], [-B, -A]] (Eq. gevpbse with Delta^2 = 1).
  * X - Y = (A-B)^{-1/2} sqrt(E) Z: the printed +1/2 power contradicts
    (A-B)(X-Y) = E (X+Y).
  * Broadening: delta is the half width (FWHM / 2).
  * Transition index alpha = (k * nv + v) * nc + c.

Parity status: build_A_B, reduce_sqrt, solve_full, oscillator_strengths and
eps_M are pinned by the tests in tests/test_oracle_pins.py (closed forms,
brute force, sum rules, gauge invariance, and the real-space double integrals
of Eq. wij for V, W^rr and W^ra, the last between a resonant and an
anti-resonant basis function built from time-reversal-symmetric Bloch
functions, which fixes the sign of W^ra in B, the conjugated N factor and the
orientation of W); block_A_B is pinned to build_A_B
block by block (tests/test_oracle_blocks.py); transition_coefficients,
eps_tensor, loss_function and structure_factor by tests/test_oracle_spectra.py
(contraction to the pinned scalar spectrum, a one-transition case worked by
hand, rotation covariance, the loss identities).
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

HARTREE_EV = 27.211386245988   # CODATA 2018


def kappa(nk: int, omega_cell: float) -> float:
    """Prefactor Ha / V_c with V_c = Nk * Omega (Eq. vft: 1/V_c; Hartree -> eV)."""
    return HARTREE_EV / (nk * omega_cell)


def transition_energies(e_v: np.ndarray, e_c: np.ndarray) -> np.ndarray:
    """E^ip_alpha = eps_c,k - eps_v,k (Eq. emat), alpha = (k, v, c)."""
    nk, nv = e_v.shape
    nc = e_c.shape[1]
    e = np.empty((nk, nv, nc))
    for k in range(nk):
        for v in range(nv):
            for c in range(nc):
                e[k, v, c] = e_c[k, c] - e_v[k, v]
    return e.reshape(-1)


def exchange_V(m_x: np.ndarray, v_bar: np.ndarray, kap: float) -> np.ndarray:
    """V^rr_{alpha alpha'} = kappa sum_G vbar_G conj(M_alpha(G)) M_alpha'(G)
    (Eq. vrrofM with the bare v replaced by vbar, Eq. vbar_def)."""
    nk, nv, nc, ng = m_x.shape
    m = m_x.reshape(nk * nv * nc, ng)
    return kap * ((np.conj(m) * v_bar[None, :]) @ m.T)


def direct_Wrr(m_vv: np.ndarray, m_cc: np.ndarray, w: np.ndarray,
               q_minus: np.ndarray, kap: float) -> np.ndarray:
    """W^rr_{(k v c),(k' v' c')} = kappa sum_{G G'} conj(M^vv[k,k',v,v',G])
    W[q-(k,k')]_{G G'} M^cc[k,k',c,c',G']   (Eq. wrrm)."""
    nk, _, nv, _, ng = m_vv.shape
    nc = m_cc.shape[2]
    out = np.zeros((nk, nv, nc, nk, nv, nc), np.complex128)
    for k in range(nk):
        for kp in range(nk):
            wq = w[q_minus[k, kp]]
            # sum over G' first, then over G, as the equation is written
            inner = np.einsum("gh,cdh->cdg", wq, m_cc[k, kp], optimize=True)
            blk = np.einsum("avg,cdg->acvd", np.conj(m_vv[k, kp]), inner, optimize=True)
            # blk[v, c, v', c']
            out[k, :, :, kp, :, :] = blk
    n = nk * nv * nc
    return kap * out.reshape(n, n)


def direct_Wra(n_vc: np.ndarray, w: np.ndarray, q_plus: np.ndarray, kap: float) -> np.ndarray:
    """W^ra_{(k v c),(k' v' c')} = kappa sum_{G G'} conj(N^cv[k,k',c,v',G])
    W[q+(k,k')]_{G G'} N^vc[k,k',v,c',G']   (Eq. wrabar), with
    N^cv[k,k',c,v'] read as n_vc[k',k,v',c].  n_vc[k,k',v,c'](G) is the
    modified plane-wave element with the ket time-reversed,
    int phi*_{v k}(r) e^{-i(G+q)r} phi*_{c' k'}(r) dr with q = -k-k'."""
    nk, _, nv, nc, ng = n_vc.shape
    out = np.zeros((nk, nv, nc, nk, nv, nc), np.complex128)
    for k in range(nk):
        for kp in range(nk):
            wq = w[q_plus[k, kp]]
            first = np.conj(n_vc[kp, k])          # [v', c, G]
            second = n_vc[k, kp]                   # [v, c', G']
            inner = np.einsum("gh,vyh->vyg", wq, second, optimize=True)
            blk = np.einsum("xcg,vyg->vcxy", first, inner, optimize=True)
            # blk[v, c, v', c']
            out[k, :, :, kp, :, :] = blk
    n = nk * nv * nc
    return kap * out.reshape(n, n)


def build_A_B(p: Dict, gamma_x: float = 1.0, gamma_c: float = 1.0,
              coupling: bool = True) -> Tuple[np.ndarray, np.ndarray]:
    """A = E^ip + 2 gamma_x V^rr - gamma_c W^rr (Eq. diagonalblock);
    B = 2 gamma_x V^rr - gamma_c W^ra (Eq. couplingblock); B = 0 in the TDA.
    gamma_x, gamma_c per Table tab:approx."""
    kap = kappa(p["nk"], p["omega_cell"])
    e = transition_energies(p["e_v"], p["e_c"])
    V = exchange_V(p["m_x"], p["v_bar"], kap)
    Wrr = direct_Wrr(p["m_vv"], p["m_cc"], p["w"], p["q_minus"], kap)
    A = np.diag(e).astype(np.complex128) + 2.0 * gamma_x * V - gamma_c * Wrr
    if coupling:
        Wra = direct_Wra(p["n_vc"], p["w"], p["q_plus"], kap)
        B = 2.0 * gamma_x * V - gamma_c * Wra
    else:
        B = np.zeros_like(A)
    return A, B


def block_A_B(blk: Dict, gamma_x: float = 1.0, gamma_c: float = 1.0,
              coupling: bool = True) -> Tuple[np.ndarray, np.ndarray]:
    """The (k, k') block of A and B, rows (v, c) and columns (v', c'), from the
    inputs of that block alone (for sampled checks of builds too large to
    form on the CPU).  Same definitions as build_A_B, term by term:
      V    = kappa sum_G conj(M_x[k,v,c,G]) vbar_G M_x[k',v',c',G]       (Eq. vrrofM)
      W^rr = kappa sum_GG' conj(M^vv[k,k',v,v',G]) W[q-]_GG' M^cc[k,k',c,c',G']   (Eq. wrrm)
      W^ra = kappa sum_GG' conj(N^cv[k,k',c,v',G]) W[q+]_GG' N^vc[k,k',v,c',G']   (Eq. wrabar)
      A = delta_kk' E^ip + 2 gamma_x V - gamma_c W^rr;  B = 2 gamma_x V - gamma_c W^ra
    blk holds: nk, omega_cell, same_k, e_v_k [nv], e_c_k [nc], m_x_k and
    m_x_kp [nv, nc, ng], v_bar [ng], m_vv [nv, nv, ng], m_cc [nc, nc, ng],
    w_minus [ng, ng] and, with coupling, n_vc_kkp = n_vc[k, k'] and
    n_vc_kpk = n_vc[k', k] [nv, nc, ng] and w_plus [ng, ng]."""
    kap = kappa(blk["nk"], blk["omega_cell"])
    mk, mkp = blk["m_x_k"], blk["m_x_kp"]
    nv, nc, ng = mk.shape
    n = nv * nc
    # V[(v,c),(v',c')]: the G sum as a matrix product over G
    V = kap * ((np.conj(mk.reshape(n, ng)) * blk["v_bar"][None, :]) @ mkp.reshape(n, ng).T)
    # W^rr: sum over G' first (W M^cc), then over G, as the equation is written
    inner = np.einsum("gh,cdh->cdg", blk["w_minus"], blk["m_cc"], optimize=True)
    Wrr = kap * np.einsum("avg,cdg->acvd", np.conj(blk["m_vv"]), inner, optimize=True)
    A = 2.0 * gamma_x * V - gamma_c * Wrr.reshape(n, n)
    if blk["same_k"]:
        e = np.array([blk["e_c_k"][c] - blk["e_v_k"][v] for v in range(nv) for c in range(nc)])
        A = A + np.diag(e)
    if not coupling:
        return A, np.zeros((n, n), np.complex128)
    # W^ra: N^cv[k,k',c,v'] is n_vc[k',k,v',c] (pair swapped)
    inner = np.einsum("gh,vyh->vyg", blk["w_plus"], blk["n_vc_kkp"], optimize=True)
    Wra = kap * np.einsum("xcg,vyg->vcxy", np.conj(blk["n_vc_kpk"]), inner, optimize=True)
    B = 2.0 * gamma_x * V - gamma_c * Wra.reshape(n, n)
    return A, B


# ----------------------------------------------------------------------------
# Eq. auxham / auxevp: the half-size reduction, in its matrix-square-root form
# ----------------------------------------------------------------------------
def hermitian_sqrt(m: np.ndarray) -> np.ndarray:
    """(M)^{1/2} of a Hermitian positive-definite matrix from its eigenpairs."""
    mu, u = np.linalg.eigh(m)
    if mu.min() <= 0.0:
        raise np.linalg.LinAlgError("matrix is not positive definite")
    return (u * np.sqrt(mu)) @ u.conj().T


def reduce_sqrt(A: np.ndarray, B: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """S = (A-B)^{1/2} (A+B) (A-B)^{1/2} (Eq. auxham).  Returns S and (A-B)^{1/2}."""
    r = hermitian_sqrt(A - B)
    s = r @ (A + B) @ r
    return 0.5 * (s + s.conj().T), r


def solve_full(A: np.ndarray, B: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Exciton energies E_lambda > 0 (ascending) and X+Y (columns) of the full BSE:
    S Z = E^2 Z (Eq. auxevp); X+Y = (A-B)^{1/2} E^{-1/2} Z (reconstruction
    after Eq. auxevp)."""
    s, r = reduce_sqrt(A, B)
    e2, z = np.linalg.eigh(s)
    if e2.min() <= 0.0:
        raise np.linalg.LinAlgError("A+B is not positive definite")
    e = np.sqrt(e2)
    xpy = (r @ z) / np.sqrt(e)[None, :]
    return e, xpy


def x_minus_y(A: np.ndarray, B: np.ndarray, e: np.ndarray, xpy: np.ndarray) -> np.ndarray:
    """X-Y from (A+B)(X+Y) = E (X-Y), which follows from Eq. gevpbse."""
    return ((A + B) @ xpy) / e[None, :]


def solve_tda(A: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """TDA: A X = E X (Eq. tdaevp)."""
    return np.linalg.eigh(A)


def brute_force_eigs(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """All 2N eigenvalues of H (X;Y) = E Delta (X;Y) (Eq. gevpbse) with
    H = [[A, B], [B, A]] (Eq. Hetr): eig(Delta H), Delta = diag(1, -1)."""
    n = A.shape[0]
    dh = np.block([[A, B], [-B, -A]])
    ev = np.linalg.eigvals(dh)
    return np.sort(ev.real), np.abs(ev.imag).max() if n else 0.0


# ----------------------------------------------------------------------------
# Eq. osci, chir, epsmtensor: oscillator strengths and eps_M
# ----------------------------------------------------------------------------
def oscillator_strengths(xpy: np.ndarray, rho: np.ndarray, vc: float) -> np.ndarray:
    """|t_lambda|^2 with t_lambda = V_c^{-1/2} sum_alpha conj((X+Y)_alpha) conj(rho_alpha)
    (Eq. osci; rho_alpha = M_alpha(G=0, q), read as q.D in the optical limit)."""
    n = xpy.shape[1]
    t = np.empty(n, np.complex128)
    for lam in range(n):
        t[lam] = np.sum(np.conj(xpy[:, lam]) * np.conj(rho)) / np.sqrt(vc)
    return np.abs(t) ** 2


def eps_M(e: np.ndarray, osc: np.ndarray, omega: np.ndarray, delta: float,
          c_q: float) -> np.ndarray:
    """eps_M(omega) = 1 - c_Q sum_lambda |t_lambda|^2 [1/(w - E + i d) + 1/(-w - E - i d)]
    (Eq. chir with Eq. epsmtensor for one direction; c_Q = 4 pi at Q = 0 and
    4 pi / |Q|^2 otherwise).  Energies in eV are converted to Hartree inside
    the brackets, which multiplies the sum by Ha."""
    out = np.empty(len(omega), np.complex128)
    for i, w in enumerate(omega):
        res = 1.0 / (w - e + 1j * delta) + 1.0 / (-w - e - 1j * delta)
        out[i] = 1.0 - c_q * HARTREE_EV * np.sum(osc * res)
    return out


def transition_coefficients(xpy: np.ndarray, D: np.ndarray, vc: float) -> np.ndarray:
    """t_{lambda,i} = -i V_c^{-1/2} sum_alpha conj((X+Y)_{alpha lambda}) conj(D_{alpha,i})
    for each Cartesian direction i (Eq. tlambdai, with the 1/V_c of Eq. osci);
    D [n, 3], returns [n_lambda, 3]."""
    nl, nd = xpy.shape[1], D.shape[1]
    t = np.empty((nl, nd), np.complex128)
    for lam in range(nl):
        for i in range(nd):
            t[lam, i] = -1j * np.sum(np.conj(xpy[:, lam]) * np.conj(D[:, i])) / np.sqrt(vc)
    return t


def eps_tensor(e: np.ndarray, t: np.ndarray, omega: np.ndarray, delta: float,
               c_q: float) -> np.ndarray:
    """eps^{ij}(w) = delta_ij - c_Q Ha sum_lambda t*_{lambda i} t_{lambda j}
    [1/(w - E + i d) + 1/(-w - E - i d)]   (Eq. epsmij; its second denominator
    read as -w - E - i delta, as in Eq. epsmtensor).  Returns [n_omega, 3, 3]."""
    nd = t.shape[1]
    out = np.empty((len(omega), nd, nd), np.complex128)
    for iw, w in enumerate(omega):
        res = 1.0 / (w - e + 1j * delta) + 1.0 / (-w - e - 1j * delta)
        for i in range(nd):
            for j in range(nd):
                out[iw, i, j] = (1.0 if i == j else 0.0) - c_q * HARTREE_EV * np.sum(
                    np.conj(t[:, i]) * t[:, j] * res)
    return out


def loss_function(eps: np.ndarray) -> np.ndarray:
    """Electron energy-loss function L = -Im 1/eps_M (Eq. Lofeps)."""
    return -np.imag(1.0 / eps)


def structure_factor(eps: np.ndarray, v_inv: float) -> np.ndarray:
    """Dynamical structure factor S(Q, w) = -(1/pi) v_G(q)^{-1} Im 1/eps_M(q, w)
    (the definition after the double-differential cross-section, Sec. on
    scattering spectra); v_inv = |G+q|^2 / (4 pi), the inverse Coulomb potential."""
    return -(1.0 / np.pi) * v_inv * np.imag(1.0 / eps)


def spectrum(A: np.ndarray, B: np.ndarray, p: Dict, coupling: bool = True):
    """Full chain: energies, oscillator strengths, eps_M on p['omega']."""
    vc = p["nk"] * p["omega_cell"]
    if coupling:
        e, xpy = solve_full(A, B)
    else:
        e, xpy = solve_tda(A)
    osc = oscillator_strengths(xpy, p["rho"], vc)
    eps = eps_M(e, osc, p["omega"], p["delta"], p["c_q"])
    return e, osc, eps
