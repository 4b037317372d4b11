"""Plain FP64 CPU oracle for the learned Davidson preconditioner.

TEST INFRASTRUCTURE ONLY: used by tests/ and nothing in the product path.
The preconditioner has no counterpart in the paper (it serves the iterative
lowest-exciton solve of the half-size problem of Eq. auxevp); this module
writes out, from their definitions, the quantities its GPU kernels compute:

  samples   for an exact pair (E, X+Y) of the full problem (Eq. gevpbse) and
            X-Y = (A+B)(X+Y)/E, the perturbed vectors x~+- = x+- + eps p (one
            direction p per pair) give the residuals of the two half-size
            equations
              r+ = (A+B) x~+ - E x~- = eps ((A+B) - E) p
              r- = (A-B) x~- - E x~+ = eps ((A-B) - E) p
            per transition a the gain that maps r_a best onto the step x~ - x
            is g*_a = Re(conj(r_a) (x~ - x)_a) / |r_a|^2; relative to the
            diagonal gain 1/(D_a - E) (D the diagonal of A+B or A-B) the target
            factor is c*_a = g*_a (D_a - E), weighted by |r_a|^2 / (D_a - E)^2
            normalised over the vector (c* = 1 everywhere when A is diagonal
            and B = 0: the diagonal preconditioner is then exact)
  features  [D_a - E, D'_a - E, S_a, E / 10]: this equation's diagonal, the
            other equation's, the off-diagonal row norm of A, the energy
  features10  [(D_a - E)/10, (D'_a - E)/10, S_a/10, E/100] then, per
            neighbouring momentum transfer i (up to two) whose exact X+Y of
            the same exciton is v_i: with x the vector the residual r corrects
            (X+Y for the (A+B) equation, X-Y for the other), b = r/(D - E),
            u = v_i/|v_i| times the unit phase of v_i^H x and d = u - x/|x|,
            the three values |u_a| sqrt(n), Re(conj(b_a) d_a) sqrt(n)/|b_a|
            and Im(conj(b_a) d_a) sqrt(n)/|b_a| (zero where b_a = 0)
  network   y = w3 . relu(W2 relu(W1 f + b1) + b2) + b3, factor c = 1 + y
  loss      sum_s w_s (c_s - c*_s)^2 / sum_s w_s
  gradient  backpropagation of that loss (pinned by finite differences in
            tests/test_mlp_oracle.py)
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

CLAMP = 1e-2   # eV: |D - E| is kept at least this far from zero


def _clamp(den: np.ndarray) -> np.ndarray:
    return np.where(np.abs(den) < CLAMP, np.where(den < 0, -CLAMP, CLAMP), den)


def diag_features(A: np.ndarray, B: np.ndarray):
    """Diagonals of A+B and A-B (real parts) and off-diagonal row norms of A."""
    dp = np.real(np.diag(A + B))
    dm = np.real(np.diag(A - B))
    off = A - np.diag(np.diag(A))
    s = np.sqrt(np.sum(np.abs(off) ** 2, axis=1))
    return dp, dm, s


def features(dq: np.ndarray, dother: np.ndarray, s: np.ndarray, e: float) -> np.ndarray:
    return np.stack([dq - e, dother - e, s, np.full_like(dq, e / 10.0)], axis=1)


def features10(dq: np.ndarray, dother: np.ndarray, s: np.ndarray, e: float, r: np.ndarray,
               x: np.ndarray, nbrs) -> np.ndarray:
    """The 10 features of one residual column r (length n) of energy e that
    corrects the vector x; nbrs: the neighbours' X+Y of the same exciton (0 to 2
    vectors; absent ones give zero features)."""
    n = len(r)
    cols = [(dq - e) / 10.0, (dother - e) / 10.0, s / 10.0, np.full(n, e / 100.0)]
    b = r / _clamp(dq - e)
    bm = np.abs(b)
    xn = x / np.linalg.norm(x)
    for i in range(2):
        if i >= len(nbrs):
            cols += [np.zeros(n)] * 3
            continue
        v = nbrs[i]
        z = np.vdot(v, x)                      # v^H x
        ph = z / abs(z) if abs(z) > 0 else 1.0
        u = v / np.linalg.norm(v) * ph
        d = u - xn
        rel = np.conj(b) * d
        safe = np.where(bm > 0, bm, 1.0)
        cols += [np.abs(u) * np.sqrt(n),
                 np.where(bm > 0, rel.real / safe, 0.0) * np.sqrt(n),
                 np.where(bm > 0, rel.imag / safe, 0.0) * np.sqrt(n)]
    return np.stack(cols, axis=1)


def samples(A, B, E, xpy, noise, eps):
    """Training samples (features [S, 4], target c* [S], weight [S]) ordered
    (lambda, equation +/-, transition a); noise is [n, nev], column lambda the
    direction p of pair lambda."""
    n, nev = xpy.shape
    dp, dm, s = diag_features(A, B)
    F, T, W = [], [], []
    for lam in range(nev):
        e = E[lam]
        xp = xpy[:, lam]
        xm = (A + B) @ xp / e
        pdir = noise[:, lam]
        tp = xp + eps * pdir
        tm = xm + eps * pdir
        rp = (A + B) @ tp - e * tm
        rm = (A - B) @ tm - e * tp
        for r, x, t, dq, do in ((rp, xp, tp, dp, dm), (rm, xm, tm, dm, dp)):
            step = t - x
            r2 = np.abs(r) ** 2
            gstar = np.where(r2 > 0, np.real(np.conj(r) * step) / np.where(r2 > 0, r2, 1.0), 0.0)
            den = _clamp(dq - e)
            c = gstar * den
            w = r2 / den ** 2
            w = w / w.sum() if w.sum() > 0 else w
            F.append(features(dq, do, s, e))
            T.append(c)
            W.append(w)
    return np.concatenate(F), np.concatenate(T), np.concatenate(W)


def init_params(f: int, h: int) -> Dict[str, np.ndarray]:
    return {"W1": np.zeros((h, f)), "b1": np.zeros(h), "W2": np.zeros((h, h)),
            "b2": np.zeros(h), "w3": np.zeros(h), "b3": np.zeros(1)}


def forward(p: Dict[str, np.ndarray], X: np.ndarray):
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss(p, X, c_star, w) -> float:
    y, _ = forward(p, X)
    return float(np.sum(w * (1.0 + y - c_star) ** 2) / np.sum(w))


def grad(p, X, c_star, w) -> Tuple[float, Dict[str, np.ndarray]]:
    """Loss and its gradient by backpropagation through the two ReLU layers."""
    y, (X, z1, h1, z2, h2) = forward(p, X)
    sw = np.sum(w)
    resid = 1.0 + y - c_star
    L = float(np.sum(w * resid ** 2) / sw)
    dy = 2.0 * w * resid / sw                     # dL/dy per sample
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, p["w3"]) * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return L, g


def factor(p, X) -> np.ndarray:
    """Preconditioner factor c = 1 + y."""
    return 1.0 + forward(p, X)[0]


PARAM_ORDER = ("W1", "b1", "W2", "b2", "w3", "b3")


def flatten(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], float).reshape(-1) for k in PARAM_ORDER])


def unflatten(v: np.ndarray, f: int, h: int) -> Dict[str, np.ndarray]:
    shapes = {"W1": (h, f), "b1": (h,), "W2": (h, h), "b2": (h,), "w3": (h,), "b3": (1,)}
    out, o = {}, 0
    for k in PARAM_ORDER:
        size = int(np.prod(shapes[k]))
        out[k] = np.asarray(v[o:o + size], float).reshape(shapes[k])
        o += size
    return out
