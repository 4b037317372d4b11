"""Seeded synthetic inputs for the BSE Hamiltonian build.

This module only draws numbers: band energies, plane-wave pair matrix
elements M and N, the screened interaction W_GG'(q), the k-point pair maps
q-(k,k') = k-k' and q+(k,k') = -k-k', and the Coulomb potential v(G+Q).  It
holds none of the method's arithmetic (no exchange or direct term, no
Hamiltonian, no spectrum); both the CPU oracle tests and the CUDA path take
their inputs from here.

Shapes follow the problem statement of the method:
  e_v  [nk, nv]            valence energies (eV)
  e_c  [nk, nc]            conduction energies (eV)
  m_x  [nk, nv, nc, ng]    M_{cv,k}(G, Q), exchange pair elements (Eq. vrrofM)
  m_vv [nk, nk, nv, nv, ng] M_{v'v}(G, k-k') indexed [k][k'][v][v'] (Eq. wrrm)
  m_cc [nk, nk, nc, nc, ng] M_{c'c}(G, k-k') indexed [k][k'][c][c'] (Eq. wrrm)
  n_vc [nk, nk, nv, nc, ng] N_{v c'}(G, -k-k') indexed [k][k'][v][c'] (Eq. wrabar)
  w    [nk, ng, ng]         W_GG'(q) for every q of the k grid
  q_minus, q_plus [nk, nk]  index of k-k' and -k-k' into w
  v_bar [ng]                4 pi / |G+Q|^2 with the G = 0 term removed (Eq. vbar_def)

Symmetries imposed so that A and B come out Hermitian (the paper states H
Hermitian in its time-reversal basis, Eq. Hetr):
  S1  W(q) Hermitian, strictly diagonally dominant with positive diagonal (PD)
  S2  W(-q) = conj(W(q)); W(q) real symmetric when q == -q on the grid
  S3  m_vv[k',k,v',v] = conj(m_vv[k,k',v,v']), likewise m_cc
  S4  N^{cv} is read from n_vc with the pair swapped (one array stored)

Every block is drawn from its own counter-keyed Philox stream
(numpy.random.Philox keyed by a hash of seed, array name, Q index and the
k / k' / q labels), so any block is reproducible on its own.
"""
from __future__ import annotations

import dataclasses
import hashlib
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

HARTREE_EV = 27.211386245988      # CODATA 2018, eV per Hartree
A_LAT_BOHR = 10.26                # Si lattice constant used for the FCC cell
OMEGA_CELL = A_LAT_BOHR ** 3 / 4  # FCC primitive-cell volume, bohr^3


@dataclasses.dataclass(frozen=True)
class BSEConfig:
    name: str
    grid: int                      # Gamma-centred grid n x n x n
    nv: int
    nc: int
    ng: int
    q_abs: Tuple[float, ...] = (0.0,)   # |Q| in bohr^-1 along [100]
    windows: Optional[Tuple[Tuple[int, int], ...]] = None  # per-Q (nv, nc)
    e_v_range: Tuple[float, float] = (-3.0, 0.0)
    e_c_range: Tuple[float, float] = (1.0, 4.0)
    m_decay: float = 1.0           # M(G) ~ CN(0,1) / (1 + m_decay |G|^2)
    w_decay: float = 1.0           # W_GG' off-diagonal ~ 1 / (1 + w_decay |G-G'|)
    w_diag: float = 1.0            # diagonal = w_diag * (1 + off-diagonal row sum)
    w_scale: float = 1.0           # overall scale on W
    fwhm_ev: float = 0.1
    omega_range: Tuple[float, float] = (0.0, 10.0)
    n_omega: int = 2000

    @property
    def nk(self) -> int:
        return self.grid ** 3

    def window(self, q_index: int) -> Tuple[int, int]:
        if self.windows is None:
            return self.nv, self.nc
        return self.windows[q_index]

    def n_trans(self, q_index: int = 0) -> int:
        nv, nc = self.window(q_index)
        return self.nk * nv * nc


def _c3_windows(seed: int = 3) -> Tuple[Tuple[int, int], ...]:
    rng = np.random.Generator(np.random.Philox(key=seed))
    wins = [(int(rng.integers(2, 5)), int(rng.integers(2, 7))) for _ in range(16)]
    wins[0] = (2, 2)
    wins[-1] = (4, 6)
    return tuple(wins)


# The w_scale values keep A-B and A+B positive definite (the reduction of
# Eq. auxham needs both PD): W^rr and W^ra are linear in W, and each scale
# was chosen once so that their spectral norms stay near a quarter of the
# smallest transition energy at that shape.
CONFIGS: Dict[str, BSEConfig] = {
    # 2x2x2 grid, 2x2 bands -> N = 32, NG = 59 (closed shell)
    "c1": BSEConfig("c1", grid=2, nv=2, nc=2, ng=59, w_scale=0.25),
    # 4x4x4 grid, 4x4 bands -> N = 1024, NG = 181 (closed shell)
    "c2": BSEConfig("c2", grid=4, nv=4, nc=4, ng=181, w_scale=0.25),
    # 8x8x8 grid, 16 Q along [100], uneven windows, NG = 113
    "c3": BSEConfig("c3", grid=8, nv=4, nc=6, ng=113,
                    q_abs=tuple(np.linspace(0.1, 1.5, 16).tolist()),
                    windows=_c3_windows(), w_scale=0.25),
    # core-like case: 2 flat core levels x 20 conduction bands, NG = 300
    "c4": BSEConfig("c4", grid=8, nv=2, nc=20, ng=300,
                    q_abs=(0.2, 0.3, 0.4, 0.5, 0.6),
                    e_v_range=(-400.5, -399.5), e_c_range=(1.0, 4.0),
                    m_decay=0.05, w_scale=0.25, omega_range=(395.0, 410.0)),
    # the core-like recipe on a 4x4x4 grid (N = 2,560): small enough for
    # profiling captures and quick Davidson checks, same pair-block shapes
    "c4s": BSEConfig("c4s", grid=4, nv=2, nc=20, ng=300,
                     q_abs=(0.2, 0.3, 0.4, 0.5, 0.6),
                     e_v_range=(-400.5, -399.5), e_c_range=(1.0, 4.0),
                     m_decay=0.05, w_scale=0.25, omega_range=(395.0, 410.0)),
    # molecular-crystal-like: 4x4x4 grid, 20x20 bands, NG = 500, strong off-diagonal W
    # (strong off-diagonal W with 500 plane waves: scale 0.002 keeps |W^rr| near
    # 0.7 eV, below the 1.1 eV smallest transition, as 0.25 does at c2)
    "c5": BSEConfig("c5", grid=4, nv=20, nc=20, ng=500,
                    q_abs=tuple(0.1 * i for i in range(8)),
                    w_decay=0.2, w_diag=1.05, w_scale=0.002),
    # the molecular-crystal-like recipe on a 2x2x2 grid (N = 3,200, 0.6 GB of
    # pair elements): the same pair-block and plane-wave shapes as c5 for
    # profiling captures of its kernels
    "c5s": BSEConfig("c5s", grid=2, nv=20, nc=20, ng=500,
                     q_abs=tuple(0.1 * i for i in range(8)),
                     w_decay=0.2, w_diag=1.05, w_scale=0.002),
}


# ----------------------------------------------------------------------------
# lattice and k grid
# ----------------------------------------------------------------------------
def reciprocal_vectors(ng: int, a: float = A_LAT_BOHR) -> np.ndarray:
    """First ng reciprocal-lattice vectors of the FCC cell (a BCC lattice),
    sorted by |G|^2 with ties broken lexicographically on the integer
    coordinates.  Returns [ng, 3] in bohr^-1; G = 0 is row 0."""
    b = 2.0 * np.pi / a * np.array([[-1, 1, 1], [1, -1, 1], [1, 1, -1]], float)

    def first(nmax):
        r = np.arange(-nmax, nmax + 1)
        ijk = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
        cart = ijk @ b
        # |G|^2 in units of (2 pi / a)^2 is an integer: sort on it exactly
        key2 = np.rint((cart ** 2).sum(1) * (a / (2 * np.pi)) ** 2).astype(np.int64)
        order = np.lexsort((ijk[:, 2], ijk[:, 1], ijk[:, 0], key2))
        return cart[order[:ng]]

    nmax = 3
    while True:   # grow the search cube until the selection stops changing
        g0, g1 = first(nmax), first(nmax + 2)
        if np.array_equal(g0, g1):
            return g0
        nmax += 2


def reciprocal_coords(ng: int) -> np.ndarray:
    """Integer coordinates [ng, 3] (in the reciprocal basis) of the vectors of
    reciprocal_vectors(ng), same order."""
    b = 2.0 * np.pi / A_LAT_BOHR * np.array([[-1, 1, 1], [1, -1, 1], [1, 1, -1]], float)
    return np.rint(reciprocal_vectors(ng) @ np.linalg.inv(b)).astype(np.int64)


def wavefunction_coefficients(grid: int, nv: int, nc: int, npw: int, seed: int = 20190411,
                              decay: float = 1.0) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Seeded plane-wave coefficients of nv valence and nc conduction Bloch
    functions at every k of the grid^3 grid, over the basis of the first npw
    reciprocal vectors (a closed shell, so G -> -G maps it onto itself):
    returns (cv [nk, nv, npw], cc [nk, nc, npw], basis [npw, 3] integer
    coordinates).  Complex normal coefficients damped by 1 / (1 + decay |G|^2),
    orthonormal over the nv + nc bands of each k, with the time-reversal
    relation C_{n,-k}(G) = conj(C_{n,k}(-G)) (phi_{n,-k} = phi_{n,k}^*); at
    k = -k the functions are real (C(-G) = conj(C(G)))."""
    nk = grid ** 3
    basis = reciprocal_coords(npw)
    g2 = (reciprocal_vectors(npw) ** 2).sum(1)
    damp = 1.0 / (1.0 + decay * g2)
    lut = {tuple(g): i for i, g in enumerate(basis)}
    minus = np.array([lut[tuple(-g)] for g in basis])
    _, _, neg = pair_maps(grid)
    nb = nv + nc
    coef = np.empty((nk, nb, npw), np.complex128)
    done = np.zeros(nk, bool)
    for k in range(nk):
        if done[k]:
            continue
        z = _cnormal(_rng(seed, "coefficients", k), (nb, npw)) * damp
        real_k = neg[k] == k
        if real_k:   # C(-G) = conj(C(G)): a real function
            z = 0.5 * (z + np.conj(z[:, minus]))
        # Gram-Schmidt; for a real function the overlaps are real, so keep them real
        for i in range(nb):
            for j in range(i):
                ov = np.vdot(z[j], z[i])
                z[i] -= (ov.real if real_k else ov) * z[j]
            z[i] /= np.linalg.norm(z[i])
        coef[k] = z
        coef[neg[k]] = np.conj(z[:, minus])
        done[k] = done[neg[k]] = True
    return coef[:, :nv], coef[:, nv:], basis


def k_grid(n: int) -> np.ndarray:
    """Integer coordinates [nk, 3] of the Gamma-centred n^3 grid, k = (i*n + j)*n + l."""
    r = np.arange(n)
    return np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)


def _k_index(ijk: np.ndarray, n: int) -> np.ndarray:
    ijk = np.mod(ijk, n)
    return (ijk[..., 0] * n + ijk[..., 1]) * n + ijk[..., 2]


def pair_maps(n: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """q_minus[k,k'] = index of k-k', q_plus[k,k'] = index of -k-k',
    neg[q] = index of -q, all on the n^3 grid (mod n)."""
    kk = k_grid(n)
    qm = _k_index(kk[:, None, :] - kk[None, :, :], n).astype(np.int32)
    qp = _k_index(-kk[:, None, :] - kk[None, :, :], n).astype(np.int32)
    neg = _k_index(-kk, n).astype(np.int32)
    return qm, qp, neg


# ----------------------------------------------------------------------------
# counter-keyed streams
# ----------------------------------------------------------------------------
def _key(*parts) -> int:
    h = hashlib.blake2b(repr(parts).encode(), digest_size=16).digest()
    return int.from_bytes(h, "little")


def _rng(*parts) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=_key(*parts)))


def _cnormal(rng: np.random.Generator, shape) -> np.ndarray:
    """Complex normal with Re and Im each N(0, 1/2)."""
    x = rng.standard_normal(shape + (2,))
    return (x[..., 0] + 1j * x[..., 1]) * np.sqrt(0.5)


# ----------------------------------------------------------------------------
# the problem
# ----------------------------------------------------------------------------
def _hermitian_pair_array(nk: int, nb: int, ng: int, damp: np.ndarray, seed, name, qi,
                          k_rows: Sequence[int]) -> np.ndarray:
    """[len(k_rows), nk, nb, nb, ng] with X[k',k,b',b] = conj(X[k,k',b,b']) (S3)."""
    out = np.empty((len(k_rows), nk, nb, nb, ng), np.complex128)
    for r, k in enumerate(k_rows):
        for kp in range(nk):
            lo, hi = (k, kp) if k <= kp else (kp, k)
            blk = _cnormal(_rng(seed, name, qi, lo, hi), (nb, nb, ng)) * damp
            if k == kp:
                iu = np.triu_indices(nb, 1)
                h = blk.copy()
                h[iu[1], iu[0]] = np.conj(blk[iu[0], iu[1]])
                d = np.arange(nb)
                h[d, d] = blk[d, d].real
                out[r, kp] = h
            elif k < kp:
                out[r, kp] = blk
            else:
                out[r, kp] = np.conj(blk.transpose(1, 0, 2))
    return out


def _w_matrix(rng, gvec, w_decay, w_diag, real):
    ng = len(gvec)
    dg = np.linalg.norm(gvec[:, None, :] - gvec[None, :, :], axis=-1)
    z = _cnormal(rng, (ng, ng))
    if real:
        z = z.real.astype(np.complex128)
    off = z / (1.0 + w_decay * dg)
    iu = np.triu_indices(ng, 1)
    w = np.zeros((ng, ng), np.complex128)
    w[iu] = off[iu]
    w[iu[1], iu[0]] = np.conj(off[iu])
    rowsum = np.abs(w).sum(1)
    w[np.arange(ng), np.arange(ng)] = w_diag * (1.0 + rowsum)
    return w


def make_problem(cfg: BSEConfig | str, q_index: int = 0, seed: int = 20190411,
                 k_rows: Optional[Sequence[int]] = None,
                 draws_of: Optional[int] = None) -> Dict[str, np.ndarray]:
    """Draw one BSE problem (one momentum transfer Q) of configuration cfg.

    k_rows restricts the pair arrays (m_vv, m_cc, n_vc) to a slab of k rows;
    every other array is always complete.  draws_of = j takes every random
    array (energies, M, N, W) from the streams of Q index j while Q itself is
    cfg.q_abs[q_index]: the problems of one j then form a family that changes
    smoothly along Q (through v(G+Q) and c_Q only), as an exciton dispersion
    needs.  Returns plain numpy arrays plus scalars: omega_cell (bohr^3), nk,
    nv, nc, ng, q_vec, c_q, rho, omega, delta (half width at half maximum,
    eV)."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    n, nk = cfg.grid, cfg.nk
    nv, nc = cfg.window(q_index)
    qd = q_index if draws_of is None else draws_of
    ng = cfg.ng
    if k_rows is None:
        k_rows = range(nk)
    k_rows = list(k_rows)

    gvec = reciprocal_vectors(ng)
    qvec = np.array([cfg.q_abs[q_index], 0.0, 0.0])
    g2 = (gvec ** 2).sum(1)
    damp = 1.0 / (1.0 + cfg.m_decay * g2)

    r_e = _rng(seed, "energies", qd)
    e_v = r_e.uniform(*cfg.e_v_range, size=(nk, nv))
    e_c = r_e.uniform(*cfg.e_c_range, size=(nk, nc))

    m_x = np.empty((nk, nv, nc, ng), np.complex128)
    for k in range(nk):
        m_x[k] = _cnormal(_rng(seed, "m_x", qd, k), (nv, nc, ng)) * damp

    m_vv = _hermitian_pair_array(nk, nv, ng, damp, seed, "m_vv", qd, k_rows)
    m_cc = _hermitian_pair_array(nk, nc, ng, damp, seed, "m_cc", qd, k_rows)
    n_vc = np.empty((len(k_rows), nk, nv, nc, ng), np.complex128)
    for r, k in enumerate(k_rows):
        for kp in range(nk):
            n_vc[r, kp] = _cnormal(_rng(seed, "n_vc", qd, k, kp), (nv, nc, ng)) * damp

    q_minus, q_plus, neg = pair_maps(n)
    w = np.empty((nk, ng, ng), np.complex128)
    for q in range(nk):
        nq = int(neg[q])
        if nq < q:
            w[q] = np.conj(w[nq])
        else:
            w[q] = _w_matrix(_rng(seed, "w", qd, q), gvec, cfg.w_decay, cfg.w_diag,
                             real=(nq == q))
    w *= cfg.w_scale

    gq = gvec + qvec[None, :]
    gq2 = (gq ** 2).sum(1)
    v_bar = np.zeros(ng)
    v_bar[1:] = 4.0 * np.pi / gq2[1:]          # G = 0 term removed (Eq. vbar_def)

    qabs = float(np.linalg.norm(qvec))
    c_q = 4.0 * np.pi if qabs == 0.0 else 4.0 * np.pi / qabs ** 2
    rho = m_x[..., 0].reshape(-1).copy()        # M_alpha(G = 0): q.D at Q = 0

    fwhm = cfg.fwhm_ev
    omega = np.linspace(cfg.omega_range[0], cfg.omega_range[1], cfg.n_omega)
    return dict(
        e_v=e_v, e_c=e_c, m_x=m_x, m_vv=m_vv, m_cc=m_cc, n_vc=n_vc, w=w,
        q_minus=q_minus, q_plus=q_plus, v_bar=v_bar, gvec=gvec, q_vec=qvec,
        omega_cell=OMEGA_CELL, nk=nk, nv=nv, nc=nc, ng=ng, k_rows=np.array(k_rows),
        c_q=c_q, rho=rho, omega=omega, delta=fwhm / 2.0,
    )


# ----------------------------------------------------------------------------
# full-size problems drawn on a device (torch)
# ----------------------------------------------------------------------------
def _torch_gen(device, *parts):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(_key(*parts) % (1 << 62))
    return g


def _hermitian_pair_torch(nk, nb, ng, damp, gen, device):
    """[nk, nk, nb, nb, ng] complex normal x damp with S3 imposed in place:
    blocks k < k' drawn, blocks k > k' their conjugate transposes (b <-> b'),
    diagonal blocks Hermitian in (b, b') with a real diagonal."""
    import torch
    x = torch.randn((nk, nk, nb, nb, ng), dtype=torch.complex128, device=device, generator=gen)
    x *= damp
    iu = torch.triu_indices(nb, nb, 1, device=device)
    d = torch.arange(nb, device=device)
    for k in range(nk):
        if k > 0:
            x[k, :k] = x[:k, k].transpose(1, 2).conj()
        blk = x[k, k]
        blk[iu[1], iu[0]] = blk[iu[0], iu[1]].conj()
        blk[d, d] = blk[d, d].real.to(torch.complex128)
    return x


def pair_slab_torch(cfg: BSEConfig | str, k_begin: int, k_count: int, q_index: int = 0,
                    seed: int = 20190411, device="cuda", draws_of: Optional[int] = None):
    """m_vv and m_cc for the k rows [k_begin, k_begin + k_count) only, drawn on
    a torch device: ([k_count, nk, nv, nv, ng], [k_count, nk, nc, nc, ng]).

    For problems whose pair arrays exceed the device memory (hundreds of GB),
    built a slab of k rows at a time.  Each block (k, k') with k <= k' is drawn
    from its own stream keyed by (seed, array, Q, k, k'); a block with k > k'
    is the conjugate transpose (b <-> b') of block (k', k), and a diagonal block
    is Hermitian in (b, b') with a real diagonal.  So S3 holds across slabs and
    any slab is reproducible on its own (the numbers differ from those of
    make_problem_torch's whole arrays).  draws_of as for make_problem_torch."""
    import torch
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    nk, ng = cfg.nk, cfg.ng
    nv, nc = cfg.window(q_index)
    qd = q_index if draws_of is None else draws_of
    gvec = reciprocal_vectors(ng)
    damp = torch.as_tensor(1.0 / (1.0 + cfg.m_decay * (gvec ** 2).sum(1)), device=device)
    gen = torch.Generator(device=device)
    out = []
    for name, nb in (("m_vv", nv), ("m_cc", nc)):
        x = torch.empty((k_count, nk, nb, nb, ng), dtype=torch.complex128, device=device)
        iu = torch.triu_indices(nb, nb, 1, device=device)
        d = torch.arange(nb, device=device)
        for r in range(k_count):
            k = k_begin + r
            for kp in range(nk):
                lo, hi = (k, kp) if k <= kp else (kp, k)
                gen.manual_seed(_key(seed, name, qd, lo, hi, "slab") % (1 << 62))
                blk = torch.randn((nb, nb, ng), dtype=torch.complex128, device=device, generator=gen)
                blk *= damp
                if k == kp:
                    blk[iu[1], iu[0]] = blk[iu[0], iu[1]].conj()
                    blk[d, d] = blk[d, d].real.to(torch.complex128)
                elif k > kp:
                    blk = blk.transpose(0, 1).conj()
                x[r, kp] = blk
        out.append(x)
    return tuple(out)


def make_problem_torch(cfg: BSEConfig | str, q_index: int = 0, seed: int = 20190411,
                       device="cuda", k_slab: Optional[Tuple[int, int]] = None,
                       draws_of: Optional[int] = None) -> Dict:
    """Draw a full-size problem directly on a torch device, for shapes whose
    inputs are too large to draw on the host (tens of GB).  Same recipe as
    make_problem (distributions, damping, W(q) construction, symmetries S1-S4,
    pair maps, v_bar, rho), but the numbers come from torch's generator, so
    they differ from make_problem's; a check copies the blocks it needs back
    to the host.  Array entries are torch tensors on `device`.

    k_slab = (k_begin, k_count) draws m_vv and m_cc for those k rows only
    (pair_slab_torch); every other array is whole.  draws_of = j draws every
    random array from the streams of Q index j (a family along Q, as in
    make_problem)."""
    import torch
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    n, nk = cfg.grid, cfg.nk
    nv, nc = cfg.window(q_index)
    qd = q_index if draws_of is None else draws_of
    ng = cfg.ng
    gvec = reciprocal_vectors(ng)
    qvec = np.array([cfg.q_abs[q_index], 0.0, 0.0])
    g2 = (gvec ** 2).sum(1)
    damp = torch.as_tensor(1.0 / (1.0 + cfg.m_decay * g2), device=device)

    ge = _torch_gen(device, seed, "energies", qd, "torch")
    lo_v, hi_v = cfg.e_v_range
    lo_c, hi_c = cfg.e_c_range
    e_v = lo_v + (hi_v - lo_v) * torch.rand((nk, nv), dtype=torch.float64, device=device, generator=ge)
    e_c = lo_c + (hi_c - lo_c) * torch.rand((nk, nc), dtype=torch.float64, device=device, generator=ge)

    m_x = torch.randn((nk, nv, nc, ng), dtype=torch.complex128, device=device,
                      generator=_torch_gen(device, seed, "m_x", qd, "torch"))
    m_x *= damp
    if k_slab is None:
        m_vv = _hermitian_pair_torch(nk, nv, ng, damp, _torch_gen(device, seed, "m_vv", qd, "torch"), device)
        m_cc = _hermitian_pair_torch(nk, nc, ng, damp, _torch_gen(device, seed, "m_cc", qd, "torch"), device)
    else:
        m_vv, m_cc = pair_slab_torch(cfg, k_slab[0], k_slab[1], q_index, seed, device, draws_of)
    n_vc = torch.randn((nk, nk, nv, nc, ng), dtype=torch.complex128, device=device,
                       generator=_torch_gen(device, seed, "n_vc", qd, "torch"))
    n_vc *= damp

    q_minus, q_plus, neg = pair_maps(n)
    gv = torch.as_tensor(gvec, device=device)
    dg = torch.cdist(gv, gv)
    gw = _torch_gen(device, seed, "w", qd, "torch")
    w = torch.empty((nk, ng, ng), dtype=torch.complex128, device=device)
    iu = torch.triu_indices(ng, ng, 1, device=device)
    d = torch.arange(ng, device=device)
    for q in range(nk):
        nq = int(neg[q])
        if nq < q:
            w[q] = w[nq].conj()
            continue
        z = torch.randn((ng, ng), dtype=torch.complex128, device=device, generator=gw)
        if nq == q:
            z = z.real.to(torch.complex128)
        off = z / (1.0 + cfg.w_decay * dg)
        wq = torch.zeros((ng, ng), dtype=torch.complex128, device=device)
        wq[iu[0], iu[1]] = off[iu[0], iu[1]]
        wq[iu[1], iu[0]] = off[iu[0], iu[1]].conj()
        wq[d, d] = (cfg.w_diag * (1.0 + wq.abs().sum(1))).to(torch.complex128)
        w[q] = wq
    w *= cfg.w_scale

    gq2 = ((gvec + qvec[None, :]) ** 2).sum(1)
    v_bar = np.zeros(ng)
    v_bar[1:] = 4.0 * np.pi / gq2[1:]          # G = 0 term removed (Eq. vbar_def)
    qabs = float(np.linalg.norm(qvec))
    c_q = 4.0 * np.pi if qabs == 0.0 else 4.0 * np.pi / qabs ** 2
    omega = np.linspace(cfg.omega_range[0], cfg.omega_range[1], cfg.n_omega)
    return dict(
        e_v=e_v, e_c=e_c, m_x=m_x, m_vv=m_vv, m_cc=m_cc, n_vc=n_vc, w=w,
        q_minus=torch.as_tensor(q_minus, device=device), q_plus=torch.as_tensor(q_plus, device=device),
        v_bar=torch.as_tensor(v_bar, device=device), gvec=gvec, q_vec=qvec,
        omega_cell=OMEGA_CELL, nk=nk, nv=nv, nc=nc, ng=ng,
        c_q=c_q, rho=m_x[..., 0].reshape(-1).clone(), omega=omega, delta=cfg.fwhm_ev / 2.0,
    )


def block_inputs(p: Dict, k: int, kp: int, coupling: bool = True) -> Dict:
    """The inputs of the (k, k') block of A and B as host numpy arrays (from a
    problem of numpy arrays or torch tensors): what a per-block check needs."""
    def h(x):
        return x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)
    qm = int(h(p["q_minus"][k, kp]))
    out = dict(nk=p["nk"], omega_cell=p["omega_cell"], same_k=(k == kp),
               e_v_k=h(p["e_v"][k]), e_c_k=h(p["e_c"][k]), m_x_k=h(p["m_x"][k]),
               m_x_kp=h(p["m_x"][kp]), v_bar=h(p["v_bar"]), m_vv=h(p["m_vv"][k, kp]),
               m_cc=h(p["m_cc"][k, kp]), w_minus=h(p["w"][qm]))
    if coupling:
        qp = int(h(p["q_plus"][k, kp]))
        out.update(n_vc_kkp=h(p["n_vc"][k, kp]), n_vc_kpk=h(p["n_vc"][kp, k]), w_plus=h(p["w"][qp]))
    return out


def scaled(problem: Dict[str, np.ndarray], **factors) -> Dict[str, np.ndarray]:
    """Copy of a problem with some arrays multiplied by scalars, e.g.
    scaled(p, w=0.0, v_bar=0.0) for the independent-particle limit."""
    out = dict(problem)
    for name, f in factors.items():
        out[name] = problem[name] * f
    return out


def directions(n: int, m: int, seed: int = 7, name: str = "directions") -> np.ndarray:
    """m seeded complex-normal unit vectors of length n, as an [n, m] array
    (perturbation directions for preconditioner training samples)."""
    out = np.empty((n, m), np.complex128)
    for j in range(m):
        v = _cnormal(_rng(seed, name, j), (n,))
        out[:, j] = v / np.linalg.norm(v)
    return out
