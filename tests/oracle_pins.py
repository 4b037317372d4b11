"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, each independent of the oracle's own formulas.  Every pin takes the
oracle module (or a stand-in with the same functions) so that
test_oracle_mutants.py can plant mistakes in a copy and see a pin fail.

  pin_ip_limit          W = v = 0: eigenvalues are E_c - E_v (Eq. emat / diagonalblock)
  pin_ip_spectrum       gamma_x = gamma_c = 0: eps_M is a closed Lorentzian sum (Eq. chir, osci)
  pin_tda               B = 0: E = eig(A) (Eq. tdaevp) and S = A^2 (Eq. auxham)
  pin_brute_force       eig of Delta H equals +-sqrt(eig S) (Eq. gevpbse vs auxevp)
  pin_real_case         real inputs: B real symmetric, eig([[A,B],[-B*,-A*]]) = +-E
  pin_rank1_rpa         one plane wave, gamma_c = 0: E solves a secular equation
  pin_sum_rules         sum E|t|^2 and sum |t|^2/E from completeness (Eq. osci + auxevp)
  pin_type3_gevp        E^2 from the generalized problem (A-B)(A+B) x = E^2 x, no square root
  pin_xmy               (A-B)(X-Y) = E (X+Y) and (X+Y)^H (X-Y) = 1
  pin_gauge_tda         complex unitary rotation of degenerate bands: A' = U^H A U
  pin_gauge_full        real orthogonal rotation: A' = U^T A U, B' = U^T B U
  pin_real_space        V and W^rr as the real-space double integrals of Eqs. vij, wij
  pin_real_space_wra    W^ra (B) as Eq. wij between a resonant and an anti-resonant
                        basis function, with time-reversal-symmetric Bloch functions
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

import bse_inputs as bi

HA = 27.211386245988


def _small(seed=7, grid=2, nv=2, nc=2, ng=15, w_scale=0.25):
    cfg = bi.BSEConfig("pin", grid=grid, nv=nv, nc=nc, ng=ng, w_scale=w_scale,
                       n_omega=400)
    return bi.make_problem(cfg, seed=seed)


def pin_ip_limit(O):
    p = bi.scaled(_small(), w=0.0, v_bar=0.0)
    A, B = O.build_A_B(p)
    e, _ = O.solve_full(A, B)
    ref = np.sort((p["e_c"][:, None, :] - p["e_v"][:, :, None]).reshape(-1))
    assert np.allclose(np.sort(e), ref, rtol=0, atol=1e-12), "W=v=0 must give E_c - E_v"


def pin_ip_spectrum(O):
    p = _small()
    A, B = O.build_A_B(p, gamma_x=0.0, gamma_c=0.0)
    e, osc, eps = O.spectrum(A, B, p)
    # closed form: poles at E_c - E_v with weights |rho|^2 / V_c
    et = (p["e_c"][:, None, :] - p["e_v"][:, :, None]).reshape(-1)
    vc = p["nk"] * p["omega_cell"]
    wgt = np.abs(p["rho"]) ** 2 / vc
    w = p["omega"][:, None]
    d = p["delta"]
    ref = 1.0 - p["c_q"] * HA * np.sum(
        wgt[None, :] * (1.0 / (w - et[None, :] + 1j * d) - 1.0 / (w + et[None, :] + 1j * d)), 1)
    assert np.allclose(eps, ref, rtol=1e-12, atol=1e-12), "IP spectrum closed form"
    # Im eps >= 0 for omega > 0 (absorption)
    assert (eps.imag[p["omega"] > 0] > 0).all()


def pin_tda(O):
    p = _small()
    A, B0 = O.build_A_B(p, coupling=False)
    assert np.abs(B0).max() == 0.0
    e, x = O.solve_tda(A)
    assert np.allclose(np.sort(e), np.sort(np.linalg.eigvalsh(A)), atol=1e-12)
    s, _ = O.reduce_sqrt(A, np.zeros_like(A))
    assert np.allclose(s, A @ A, atol=1e-11), "S = A^2 when B = 0"
    ef, _ = O.solve_full(A, np.zeros_like(A))
    assert np.allclose(ef, np.sort(e), atol=1e-11), "full with B = 0 equals TDA"


def pin_brute_force(O):
    p = _small()
    A, B = O.build_A_B(p)
    e, _ = O.solve_full(A, B)
    ev, imag = O.brute_force_eigs(A, B)
    assert imag < 1e-9, "Delta H must have a real spectrum when A +- B are PD"
    n = len(e)
    assert np.allclose(ev[n:], e, atol=1e-10)
    assert np.allclose(ev[:n], -e[::-1], atol=1e-10), "+-E pairs (Eq. resolventwithev)"
    # independent of the oracle: numpy's general eigensolver on the 2N block form
    H = np.block([[A, B], [B, A]])
    D = np.diag(np.r_[np.ones(n), -np.ones(n)])
    ev2 = np.sort(scipy.linalg.eigvals(H, D).real)
    assert np.allclose(ev2, ev, atol=1e-10)


def pin_real_case(O):
    p = _small()
    for name in ("m_x", "m_vv", "m_cc", "n_vc", "w"):
        p[name] = p[name].real.astype(np.complex128)
    # keep the real n_vc consistent with S4 symmetry requirements (none needed)
    A, B = O.build_A_B(p)
    assert np.abs(B - B.T).max() < 1e-13, "real case: B symmetric"
    assert np.abs(A.imag).max() == 0.0 and np.abs(B.imag).max() == 0.0
    e, _ = O.solve_full(A, B)
    H = np.block([[A, B], [-B.conj(), -A.conj()]])
    ev = np.sort(np.linalg.eigvals(H).real)
    n = len(e)
    assert np.allclose(ev[n:], e, atol=1e-10) and np.allclose(ev[:n], -e[::-1], atol=1e-10)


def _secular_roots(e_a, wgt, c):
    """Roots lambda of f(lambda) = 1 - c sum_a e_a w_a / (lambda - e_a^2) = 0.
    f rises from -inf to +inf between consecutive poles e_a^2 and from -inf
    to 1 above the last one, so each interval holds one root: bisection."""
    order = np.argsort(e_a)
    e_a, wgt = e_a[order], wgt[order]
    poles = e_a ** 2
    f = lambda lam: 1.0 - c * np.sum(e_a * wgt / (lam - poles))
    upper = poles[-1] + c * np.sum(e_a * wgt) + 1.0
    roots = []
    for lo, hi in list(zip(poles[:-1], poles[1:])) + [(poles[-1], upper)]:
        for _ in range(2000):
            m = 0.5 * (lo + hi)
            if m <= lo or m >= hi:
                break
            if f(m) < 0.0:
                lo = m
            else:
                hi = m
        roots.append(0.5 * (lo + hi))
    return np.sqrt(np.array(roots))


def pin_rank1_rpa(O):
    # one plane wave with potential v, exchange only (RPA row of Table tab:approx)
    rng = np.random.default_rng(11)
    nv, nc = 2, 3
    p = _small(grid=2, nv=nv, nc=nc, ng=1)
    nk = p["nk"]
    p["e_v"] = rng.uniform(-3, 0, (nk, nv))
    p["e_c"] = rng.uniform(1, 4, (nk, nc))
    p["m_x"] = (rng.standard_normal((nk, nv, nc, 1)) + 1j * rng.standard_normal((nk, nv, nc, 1)))
    p["v_bar"] = np.array([3.7])
    A, B = O.build_A_B(p, gamma_x=1.0, gamma_c=0.0)
    e, _ = O.solve_full(A, B)
    ea = (p["e_c"][:, None, :] - p["e_v"][:, :, None]).reshape(-1)
    kap = HA / (nk * p["omega_cell"])     # 1 / V_c, V_c = Nk * Omega (Eq. vft)
    m2 = np.abs(p["m_x"].reshape(-1)) ** 2
    ref = _secular_roots(ea, m2, 4.0 * kap * 3.7)
    assert np.allclose(np.sort(e), np.sort(ref), rtol=1e-11, atol=1e-11), "rank-1 RPA secular roots"


def pin_sum_rules(O):
    p = _small()
    A, B = O.build_A_B(p)
    e, osc, _ = O.spectrum(A, B, p)
    vc = p["nk"] * p["omega_cell"]
    rt = np.conj(p["rho"])
    s1 = np.real(rt.conj() @ (A - B) @ rt) / vc
    s2 = np.real(rt.conj() @ np.linalg.solve(A + B, rt)) / vc
    assert np.isclose(np.sum(e * osc), s1, rtol=1e-11), "sum E |t|^2 = rho^H (A-B) rho / V_c"
    assert np.isclose(np.sum(osc / e), s2, rtol=1e-11), "sum |t|^2 / E = rho^H (A+B)^-1 rho / V_c"


def pin_type3_gevp(O):
    p = _small()
    A, B = O.build_A_B(p)
    e, _ = O.solve_full(A, B)
    e2 = scipy.linalg.eigh(A + B, A - B, type=3, eigvals_only=True)
    assert np.allclose(np.sort(e2), e ** 2, rtol=1e-11)
    # and the Cholesky form used by a GPU solver: A-B = L L^H, S = L^H (A+B) L
    L = np.linalg.cholesky(A - B)
    e2c = np.linalg.eigvalsh(L.conj().T @ (A + B) @ L)
    assert np.allclose(np.sort(e2c), e ** 2, rtol=1e-11)


def pin_xmy(O):
    p = _small()
    A, B = O.build_A_B(p)
    e, xpy = O.solve_full(A, B)
    xmy = O.x_minus_y(A, B, e, xpy)
    assert np.allclose((A - B) @ xmy, xpy * e[None, :], atol=1e-10)
    assert np.allclose(xpy.conj().T @ xmy, np.eye(len(e)), atol=1e-10)
    # Eq. gevpbse itself: H (X;Y) = E Delta (X;Y)
    x, y = 0.5 * (xpy + xmy), 0.5 * (xpy - xmy)
    H = np.block([[A, B], [B, A]])
    lhs = H @ np.vstack([x, y])
    rhs = np.vstack([x, -y]) * e[None, :]
    assert np.allclose(lhs, rhs, atol=1e-10)


def _random_unitary(rng, n, real):
    z = rng.standard_normal((n, n))
    if not real:
        z = z + 1j * rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def _gauge_case(O, real):
    """Rotate degenerate valence (U^k) and conduction (R^k) states at every k.
    With |n k> -> sum_a X_{a n} |a k>, a matrix element <bra|e^{-i(G+q)r}|ket>
    picks up conj(X_bra) on the bra index and X_ket on the ket index:
      m_x[k][v][c]       = <c k | . | v k>     (Eq. vrrofM: M_{u o k})
      m_vv[k][k'][v][v'] = <v' k' | . | v k>   (Eq. wrrm: M_{o' o k'})
      m_cc[k][k'][c][c'] = <c' k' | . | c k>   (Eq. wrrm: M_{u' u k'})
      n_vc[k][k'][v][c'] = <v k | . | c' k'>   (Eq. wrabar, time reversal)
    The transition (o, u, k) transforms as phi_o phi_u^* (Eq.
    2particlebasis_qsym_res): T_{(a b k),(v c k)} = U^k_{a v} conj(R^k_{b c})."""
    rng = np.random.default_rng(5 if real else 6)
    p = _small(nv=2, nc=3, ng=9)
    nk, nv, nc = p["nk"], p["nv"], p["nc"]
    p["e_v"] = np.repeat(rng.uniform(-3, 0, (nk, 1)), nv, 1)
    p["e_c"] = np.repeat(rng.uniform(1, 4, (nk, 1)), nc, 1)
    U = [_random_unitary(rng, nv, real) for _ in range(nk)]
    R = [_random_unitary(rng, nc, real) for _ in range(nk)]
    q = dict(p)
    q["m_x"] = np.stack([np.einsum("bc,av,abg->vcg", R[k].conj(), U[k], p["m_x"][k])
                         for k in range(nk)])
    mvv = np.empty_like(p["m_vv"])
    mcc = np.empty_like(p["m_cc"])
    nvc = np.empty_like(p["n_vc"])
    for k in range(nk):
        for kp in range(nk):
            mvv[k, kp] = np.einsum("bw,av,abg->vwg", U[kp].conj(), U[k], p["m_vv"][k, kp])
            mcc[k, kp] = np.einsum("bd,ac,abg->cdg", R[kp].conj(), R[k], p["m_cc"][k, kp])
            nvc[k, kp] = np.einsum("av,bd,abg->vdg", U[k].conj(), R[kp], p["n_vc"][k, kp])
    q["m_vv"], q["m_cc"], q["n_vc"] = mvv, mcc, nvc
    n = nk * nv * nc
    T = np.zeros((n, n), np.complex128)
    for k in range(nk):
        blk = np.einsum("av,bc->abvc", U[k], R[k].conj()).reshape(nv * nc, nv * nc)
        T[k * nv * nc:(k + 1) * nv * nc, k * nv * nc:(k + 1) * nv * nc] = blk
    return p, q, T


def pin_gauge_tda(O):
    p, q, T = _gauge_case(O, real=False)
    A, _ = O.build_A_B(p, coupling=False)
    A2, _ = O.build_A_B(q, coupling=False)
    assert np.allclose(A2, T.conj().T @ A @ T, atol=1e-12), "A transforms as T^H A T"
    assert np.allclose(np.linalg.eigvalsh(A2), np.linalg.eigvalsh(A), atol=1e-12)


def pin_gauge_full(O):
    p, q, T = _gauge_case(O, real=True)
    A, B = O.build_A_B(p)
    A2, B2 = O.build_A_B(q)
    assert np.allclose(A2, T.T @ A @ T, atol=1e-12)
    assert np.allclose(B2, T.T @ B @ T, atol=1e-12), "B transforms as T^T B T"
    e, _ = O.solve_full(A, B)
    e2, _ = O.solve_full(A2, B2)
    assert np.allclose(e, e2, atol=1e-12)


ALL_PINS = [pin_ip_limit, pin_ip_spectrum, pin_tda, pin_brute_force, pin_real_case,
            pin_rank1_rpa, pin_sum_rules, pin_type3_gevp, pin_xmy, pin_gauge_tda,
            pin_gauge_full]


# ----------------------------------------------------------------------------
# real-space pin: V and W^rr as the double integrals of Eq. vij and Eq. wij
# ----------------------------------------------------------------------------
def _real_space_case(seed=3, nv=2, nc=2, ncell=3, ngrid=3, a=4.0):
    """Explicit Bloch functions phi_nk(r) = e^{ikr} u_nk(r) on the real-space
    grid of an ngrid^3 supercell of a simple-cubic cell (ncell^3 points per
    cell).  Pair densities M are the discrete crystal integrals
    <bra| e^{-i(G+q) r} |ket>; the cell G set and the k grid together cover
    one full period of the supercell grid frequencies, so the plane-wave sums
    and the real-space double sums are the same finite sums in another order."""
    rng = np.random.default_rng(seed)
    nk = ngrid ** 3
    L = ngrid * a
    nr1 = ngrid * ncell
    x = np.arange(nr1) * (L / nr1)
    r = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    vc = L ** 3
    dv = vc / len(r)
    b = 2 * np.pi / a
    gi = np.arange(ncell) - ncell // 2
    gint = np.stack(np.meshgrid(gi, gi, gi, indexing="ij"), -1).reshape(-1, 3)
    gvec = gint * b
    kint = bi.k_grid(ngrid)
    kvec = kint * (b / ngrid)
    qm, qp, neg = bi.pair_maps(ngrid)

    def bloch(k, nb):
        c = rng.standard_normal((nb, len(gvec))) + 1j * rng.standard_normal((nb, len(gvec)))
        c /= (1.0 + (gvec ** 2).sum(1))[None, :]
        u = c @ np.exp(1j * gvec @ r.T)
        return u * np.exp(1j * r @ kvec[k])[None, :]

    phv = [bloch(k, nv) for k in range(nk)]
    phc = [bloch(k, nc) for k in range(nk)]

    def melem(bra, ket, kq):           # [nb_bra?] -> <bra_i| e^{-i kq r} |ket_j>[i, j, G]
        ph = np.exp(-1j * (gvec[None, :, :] + kq[None, None, :]) @ r.T[None]).reshape(len(gvec), -1)
        return np.einsum("ir,gr,jr->ijg", bra.conj(), ph, ket) * dv

    ng = len(gvec)
    m_x = np.empty((nk, nv, nc, ng), np.complex128)
    for k in range(nk):
        m_x[k] = melem(phc[k], phv[k], np.zeros(3)).transpose(1, 0, 2)   # <c|.|v> -> [v, c]
    m_vv = np.empty((nk, nk, nv, nv, ng), np.complex128)
    m_cc = np.empty((nk, nk, nc, nc, ng), np.complex128)
    for k in range(nk):
        for kp in range(nk):
            q = kvec[qm[k, kp]]
            m_vv[k, kp] = melem(phv[kp], phv[k], q).transpose(1, 0, 2)  # <v' k'|.|v k> -> [v, v']
            m_cc[k, kp] = melem(phc[kp], phc[k], q).transpose(1, 0, 2)  # <c' k'|.|c k> -> [c, c']
    # a screened interaction with off-diagonal structure: random Hermitian w_GG'(q)
    w = np.empty((nk, ng, ng), np.complex128)
    for q in range(nk):
        z = rng.standard_normal((ng, ng)) + 1j * rng.standard_normal((ng, ng))
        w[q] = 0.5 * (z + z.conj().T) + 3.0 * np.eye(ng)
    v_bar = np.where((gvec ** 2).sum(1) > 0, 4 * np.pi / np.maximum((gvec ** 2).sum(1), 1e-300), 0.0)
    p = dict(e_v=np.zeros((nk, nv)), e_c=np.ones((nk, nc)), m_x=m_x, m_vv=m_vv, m_cc=m_cc,
             n_vc=np.zeros((nk, nk, nv, nc, ng), np.complex128), w=w,
             q_minus=qm, q_plus=qp, v_bar=v_bar, omega_cell=a ** 3, nk=nk, nv=nv, nc=nc, ng=ng)

    # Coulomb kernel v(r - r') = (1/V_c) sum_{K != 0} 4 pi / |K|^2 e^{i K (r - r')}
    # over K = G + q: one full period of the supercell grid frequencies
    K = (gvec[:, None, :] + kvec[None, :, :]).reshape(-1, 3)
    k2 = (K ** 2).sum(1)
    wk = np.where(k2 > 1e-12, 4 * np.pi / np.where(k2 > 1e-12, k2, 1.0), 0.0) / vc
    E = np.exp(1j * r @ K.T)                      # [nr, nK]
    kern = (E * wk[None, :]) @ E.conj().T         # kern[r, r'] = v(r - r')
    # w(r, r') = (1/V_c) sum_q sum_{G G'} e^{i(G+q) r} w_GG'(q) e^{-i(G'+q) r'}  (Eq. wft)
    kern_w = np.zeros_like(kern)
    for q in range(nk):
        Eq = np.exp(1j * r @ (gvec + kvec[q]).T)  # [nr, ng]
        kern_w += Eq @ w[q] @ Eq.conj().T
    kern_w /= vc
    return p, phv, phc, kern, kern_w, dv


def pin_real_space(O):
    """Eq. vij:  V_{a a'} = int int Ups*_a(r, r) v(r, r') Ups_a'(r', r')
       Eq. wij:  W_{a a'} = int int Ups*_a(r, r') w(r, r') Ups_a'(r, r')
    with Ups_a(r, r') = phi_{o k}(r) phi*_{u k}(r') (Eq. 2particlebasis_qsym_res)
    with v the bare Coulomb kernel (Eq. vft, K = 0 removed) and w built from
    random Hermitian w_GG'(q) by Eq. wft; Hartree -> eV by x Ha."""
    p, phv, phc, kern, kern_w, dv = _real_space_case()
    nk, nv, nc = p["nk"], p["nv"], p["nc"]
    n = nk * nv * nc
    # transition densities on the grid, alpha = (k, v, c)
    pair_same = np.stack([phv[k][:, None, :].conj() * phc[k][None, :, :]
                          for k in range(nk)]).reshape(n, -1)       # phi*_o(r) phi_u(r)
    V_rs = HA * dv * dv * (pair_same @ kern @ pair_same.conj().T)
    # W: [phi*_o(r) phi_o'(r)] w(r - r') [phi_u(r') phi*_u'(r')]
    W_rs = np.zeros((n, n), np.complex128)
    for k in range(nk):
        for kp in range(nk):
            d1 = (phv[k][:, None, :].conj() * phv[kp][None, :, :]).reshape(nv * nv, -1)   # [o, o']
            d2 = (phc[k][:, None, :] * phc[kp][None, :, :].conj()).reshape(nc * nc, -1)   # [u, u']
            blk = (d1 @ kern_w @ d2.T).reshape(nv, nv, nc, nc) * dv * dv * HA
            W_rs[k * nv * nc:(k + 1) * nv * nc, kp * nv * nc:(kp + 1) * nv * nc] = \
                blk.transpose(0, 2, 1, 3).reshape(nv * nc, nv * nc)
    ev = np.repeat(np.ones(nv * nc)[None], nk, 0).reshape(-1)
    A_x, _ = O.build_A_B(p, gamma_x=1.0, gamma_c=0.0, coupling=False)
    A_c, _ = O.build_A_B(p, gamma_x=0.0, gamma_c=1.0, coupling=False)
    V_or = 0.5 * (A_x - np.diag(ev))
    W_or = np.diag(ev) - A_c
    scale = np.abs(V_rs).max()
    assert np.allclose(V_or, V_rs, rtol=0, atol=1e-11 * scale), "exchange = Eq. vij integral"
    scale = np.abs(W_rs).max()
    assert np.allclose(W_or, W_rs, rtol=0, atol=1e-11 * scale), "direct = Eq. wij integral"


ALL_PINS.append(pin_real_space)


# ----------------------------------------------------------------------------
# real-space pin of the coupling block: W^ra as the double integral of Eq. wij
# between a resonant and an anti-resonant basis function
# ----------------------------------------------------------------------------
def _real_space_tr_case(seed=4, nv=2, nc=2, ncell=3, ngrid=3, a=4.0):
    """Bloch functions with time-reversal symmetry, phi_{n,-k}(r) = phi*_{n,k}(r)
    (the property the basis of Eqs. 2particlebasis_qsym_res/ares relies on),
    on the real-space grid of an ngrid^3 supercell, and a screened interaction
    w(r, r') that is symmetric in r <-> r' (as the static w of a system with
    time-reversal symmetry is), given by its Fourier components w_GG'(q) of
    Eq. wft.  Plane waves on the grid are e^{i f r} with f = G + q on the
    lattice (b / ngrid) Z^3, periodic over ncell * b: the cell G box and the k
    grid cover one period exactly, so every frequency has one (G, q) label."""
    rng = np.random.default_rng(seed)
    nk = ngrid ** 3
    L = ngrid * a
    nr1 = ngrid * ncell
    x = np.arange(nr1) * (L / nr1)
    r = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    vc = L ** 3
    dv = vc / len(r)
    b = 2 * np.pi / a
    gi = np.arange(ncell) - ncell // 2
    gint = np.stack(np.meshgrid(gi, gi, gi, indexing="ij"), -1).reshape(-1, 3)
    gvec = gint * b
    ng = len(gvec)
    kint = bi.k_grid(ngrid)
    kvec = kint * (b / ngrid)
    qm, qp, neg = bi.pair_maps(ngrid)

    # time-reversal pairs: draw phi_k for one k of each pair {k, -k} and set
    # phi_{-k} = conj(phi_k); at k = -k (the Gamma point here) phi is real
    def draw(nb, k):
        c = rng.standard_normal((nb, ng)) + 1j * rng.standard_normal((nb, ng))
        c /= (1.0 + (gvec ** 2).sum(1))[None, :]
        return (c @ np.exp(1j * gvec @ r.T)) * np.exp(1j * r @ kvec[k])[None, :]

    phv, phc = [None] * nk, [None] * nk
    for k in range(nk):
        if phv[k] is not None:
            continue
        fv, fc = draw(nv, k), draw(nc, k)
        if neg[k] == k:
            fv, fc = fv.real.astype(np.complex128), fc.real.astype(np.complex128)
        phv[k], phc[k] = fv, fc
        phv[neg[k]], phc[neg[k]] = fv.conj(), fc.conj()
    for k in range(nk):   # phi_{-k} = phi_k^* holds on the grid
        assert np.allclose(phv[neg[k]], phv[k].conj()) and np.allclose(phc[neg[k]], phc[k].conj())

    # w over grid frequencies F = ngrid * G + q (integers mod nr1): Hermitian,
    # block-diagonal in the q class, then symmetrised so that
    # w(r, r') = w(r', r), i.e. w_F,F' = w_-F',-F
    fint = (ngrid * gint[:, None, :] + kint[None, :, :]).reshape(-1, 3)      # [(G, q)]
    fidx = {tuple(np.mod(f, nr1)): i for i, f in enumerate(fint)}
    minus = np.array([fidx[tuple(np.mod(-f, nr1))] for f in fint])
    qcls = np.tile(np.arange(nk), ng)
    nf = len(fint)
    z = rng.standard_normal((nf, nf)) + 1j * rng.standard_normal((nf, nf))
    wf = 0.5 * (z + z.conj().T) + 3.0 * np.eye(nf)
    wf = np.where(qcls[:, None] == qcls[None, :], wf, 0.0)
    wf = 0.5 * (wf + wf.T[np.ix_(minus, minus)])
    assert np.allclose(wf, wf.conj().T)
    w = np.empty((nk, ng, ng), np.complex128)
    for q in range(nk):
        sel = np.arange(ng) * nk + q                 # the frequencies G + q, G in box order
        w[q] = wf[np.ix_(sel, sel)]
    fvec = fint * (b / ngrid)
    E = np.exp(1j * r @ fvec.T)                       # [nr, nf]
    kern_w = (E @ wf @ E.conj().T) / vc               # Eq. wft
    assert np.allclose(kern_w, kern_w.T, atol=1e-12 * np.abs(kern_w).max())

    # n_vc[k][k'][v][c'](G) = int phi*_{v k}(r) e^{-i (G + q) r} phi*_{c' k'}(r) dr
    # with q = q+(k, k') = -k - k' on the grid: the modified plane-wave matrix
    # element N of the LAPW section with its ket state conjugated, |(c' k')^*>
    n_vc = np.empty((nk, nk, nv, nc, ng), np.complex128)
    for k in range(nk):
        for kp in range(nk):
            qv = kvec[qp[k, kp]]
            ph = np.exp(-1j * (gvec + qv[None, :]) @ r.T)              # [ng, nr]
            n_vc[k, kp] = np.einsum("ir,gr,jr->ijg", phv[k].conj(), ph, phc[kp].conj()) * dv
    p = dict(e_v=np.zeros((nk, nv)), e_c=np.ones((nk, nc)),
             m_x=np.zeros((nk, nv, nc, ng), np.complex128),
             m_vv=np.zeros((nk, nk, nv, nv, ng), np.complex128),
             m_cc=np.zeros((nk, nk, nc, nc, ng), np.complex128),
             n_vc=n_vc, w=w, q_minus=qm, q_plus=qp, v_bar=np.zeros(ng),
             omega_cell=a ** 3, nk=nk, nv=nv, nc=nc, ng=ng)
    return p, phv, phc, neg, kern_w, dv


def pin_real_space_wra(O):
    """Eq. wij with i resonant and j anti-resonant:
         W^ra_{a a'} = int int Ups^r*_a(r, r') w(r, r') Ups^a_a'(r, r')
       Ups^r_a(r, r')  = phi_{v k}(r) phi*_{c k}(r')          (Eq. 2particlebasis_qsym_res)
       Ups^a_a'(r, r') = phi_{c', -k'}(r) phi*_{v', -k'}(r')   (Eq. 2particlebasis_qsym_ares)
    at zero momentum transfer, evaluated as a double sum on the grid with the
    anti-resonant functions taken at -k' directly; B = 2 gx V - gc W^ra
    (Eq. couplingblock) with gx = 0, gc = 1 must equal -W^ra (x Ha)."""
    p, phv, phc, neg, kern_w, dv = _real_space_tr_case()
    nk, nv, nc = p["nk"], p["nv"], p["nc"]
    n = nk * nv * nc
    W_rs = np.zeros((n, n), np.complex128)
    for k in range(nk):
        for kp in range(nk):
            km = neg[kp]
            # r: phi*_{v k}(r) phi_{c', -k'}(r);  r': phi_{c k}(r') phi*_{v', -k'}(r')
            d1 = (phv[k][:, None, :].conj() * phc[km][None, :, :]).reshape(nv * nc, -1)   # [v, c']
            d2 = (phc[k][:, None, :] * phv[km][None, :, :].conj()).reshape(nc * nv, -1)   # [c, v']
            blk = (d1 @ kern_w @ d2.T).reshape(nv, nc, nc, nv) * dv * dv * HA
            # blk[v, c', c, v'] -> rows (v, c), columns (v', c')
            W_rs[k * nv * nc:(k + 1) * nv * nc, kp * nv * nc:(kp + 1) * nv * nc] = \
                blk.transpose(0, 2, 3, 1).reshape(nv * nc, nv * nc)
    scale = np.abs(W_rs).max()
    assert np.allclose(W_rs, W_rs.conj().T, atol=1e-11 * scale), "W^ra Hermitian (time reversal)"
    _, B = O.build_A_B(p, gamma_x=0.0, gamma_c=1.0, coupling=True)
    assert np.allclose(B, -W_rs, rtol=0, atol=1e-11 * scale), "coupling block = -Eq. wij (r, a)"


ALL_PINS.append(pin_real_space_wra)
