"""Pins for the MLP oracle (CPU): the backpropagated gradient against central
finite differences of the loss, a closed form with zero hidden weights, and
the sample targets on a problem where the exact answer is known."""
import numpy as np

import bse_inputs as bi
from oracle import bse_oracle as O
from oracle import mlp_oracle as M


def _rand_params(rng, f=4, h=16, scale=0.5):
    p = M.init_params(f, h)
    for k in p:
        p[k] = rng.standard_normal(p[k].shape) * scale
    return p


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = _rand_params(rng)
    X = rng.standard_normal((40, 4))
    c = rng.standard_normal(40)
    w = rng.uniform(0.1, 1.0, 40)
    L, g = M.grad(p, X, c, w)
    assert np.isclose(L, M.loss(p, X, c, w))
    v = M.flatten(p)
    gv = M.flatten(g)
    h = 1e-6
    for idx in rng.choice(len(v), 60, replace=False):
        vp, vm = v.copy(), v.copy()
        vp[idx] += h
        vm[idx] -= h
        fd = (M.loss(M.unflatten(vp, 4, 16), X, c, w) - M.loss(M.unflatten(vm, 4, 16), X, c, w)) / (2 * h)
        assert abs(fd - gv[idx]) < 1e-6 * max(1.0, abs(fd)), idx


def test_zero_hidden_weights_closed_form():
    # W1 = W2 = 0, b1, b2 > 0: y = w3 . relu(b2) + b3, constant over samples
    p = M.init_params(4, 8)
    p["b2"] = np.linspace(0.1, 0.8, 8)
    p["w3"] = np.linspace(-1, 1, 8)
    p["b3"] = np.array([0.3])
    X = np.random.default_rng(1).standard_normal((10, 4))
    c = np.linspace(0, 2, 10)
    w = np.ones(10)
    y0 = p["w3"] @ p["b2"] + 0.3
    L, g = M.grad(p, X, c, w)
    assert np.allclose(M.forward(p, X)[0], y0)
    assert np.isclose(L, np.mean((1 + y0 - c) ** 2))
    assert np.isclose(g["b3"][0], 2 * np.mean(1 + y0 - c))
    assert np.allclose(g["w3"], 2 * np.mean(1 + y0 - c) * p["b2"])


def test_sample_targets_diagonal_problem():
    # B = 0 and A diagonal: X+Y = X-Y are unit vectors and both residuals are
    # eps (D - E) p, so the diagonal gain maps them onto the step exactly:
    # c* = 1 wherever the residual is non-zero (a != lambda)
    rng = np.random.default_rng(2)
    n, nev = 12, 3
    d = np.sort(rng.uniform(1, 5, n))
    A = np.diag(d).astype(complex)
    B = np.zeros_like(A)
    E, xpy = O.solve_full(A, B)
    E, xpy = E[:nev], xpy[:, :nev]
    noise = (rng.standard_normal((n, nev)) + 1j * rng.standard_normal((n, nev)))
    F, c, w = M.samples(A, B, E, xpy, noise, 1e-3)
    # the component of the eigenvector itself has D - E = 0 (clamped): skip those
    lam = np.repeat(np.arange(nev), 2 * n)
    a = np.tile(np.arange(n), 2 * nev)
    mask = a != lam
    assert np.allclose(c[mask], 1.0, atol=1e-9)
    assert np.all(w[~mask] < 1e-15)
    assert np.allclose(F[:, 0], F[:, 1])                 # D+ = D- when B = 0
    assert np.allclose(F[:, 2], 0.0)                     # no off-diagonal coupling


def _feat10_case(rng, n=37):
    dq = rng.uniform(3, 9, n)
    do = dq + rng.uniform(-0.5, 0.5, n)
    s = rng.uniform(0, 4, n)
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v1 = x + 0.3 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    v2 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return dq, do, s, 2.5, r, x, [v1, v2]


def test_features10_by_hand():
    # one transition worked out from the definition with plain scalars
    rng = np.random.default_rng(5)
    dq, do, s, e, r, x, nb = _feat10_case(rng, n=5)
    F = M.features10(dq, do, s, e, r, x, nb)
    a = 3
    assert np.isclose(F[a, 0], (dq[a] - e) / 10) and np.isclose(F[a, 3], e / 100)
    v = nb[1]
    z = sum(np.conj(v[i]) * x[i] for i in range(5))
    u_a = v[a] / np.sqrt(sum(abs(t) ** 2 for t in v)) * z / abs(z)
    d_a = u_a - x[a] / np.sqrt(sum(abs(t) ** 2 for t in x))
    b_a = r[a] / (dq[a] - e)
    rel = np.conj(b_a) * d_a / abs(b_a) * np.sqrt(5)
    assert np.allclose(F[a, 7:10], [abs(u_a) * np.sqrt(5), rel.real, rel.imag])


def test_features10_invariances():
    rng = np.random.default_rng(6)
    dq, do, s, e, r, x, nb = _feat10_case(rng)
    F = M.features10(dq, do, s, e, r, x, nb)
    # a common phase of (r, x) and any phase of a neighbour vector change nothing
    ph = np.exp(0.7j)
    F2 = M.features10(dq, do, s, e, r * ph, x * ph, [nb[0] * np.exp(-1.1j), nb[1] * 1j])
    assert np.allclose(F, F2)
    # the scale of x and of the neighbours changes nothing either
    F3 = M.features10(dq, do, s, e, r, 3.0 * x, [0.5 * nb[0], 7.0 * nb[1]])
    assert np.allclose(F, F3)


def test_features10_special_cases():
    rng = np.random.default_rng(7)
    dq, do, s, e, r, x, nb = _feat10_case(rng)
    # a neighbour equal to the current vector: u = x/|x|, d = 0
    F = M.features10(dq, do, s, e, r, x, [x.copy()])
    assert np.allclose(F[:, 4], np.abs(x) / np.linalg.norm(x) * np.sqrt(len(x)))
    assert np.allclose(F[:, 5:7], 0.0)
    assert np.allclose(F[:, 7:], 0.0)            # no second neighbour
    # a zero residual component: its direction features are zero
    r0 = r.copy()
    r0[4] = 0
    F0 = M.features10(dq, do, s, e, r0, x, nb)
    assert np.allclose(F0[4, [5, 6, 8, 9]], 0.0)
    # sum over a of |u_a|^2 n / n = 1 (u is a unit vector)
    F1 = M.features10(dq, do, s, e, r, x, nb)
    assert np.isclose(np.sum(F1[:, 4] ** 2) / len(x), 1.0)
