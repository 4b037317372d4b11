"""The RPA screening oracle (oracle/rpa_oracle.py) against its pins (CPU):
closed forms worked by hand and identities the definition must satisfy."""
import numpy as np

from oracle import rpa_oracle as R
from oracle.bse_oracle import kappa

OMEGA = 270.0


def _case(seed=3, nk=2, nv=2, nc=3, ng=6):
    rng = np.random.default_rng(seed)
    e_v = rng.uniform(-3.0, 0.0, (nk, nv))
    e_c = rng.uniform(1.0, 4.0, (nk, nc))
    m = (rng.standard_normal((nk, nv, nc, ng)) + 1j * rng.standard_normal((nk, nv, nc, ng))) * 0.7
    v_g = rng.uniform(0.5, 3.0, ng)
    return e_v, e_c, m, v_g


def test_no_transitions_leave_the_bare_potential():
    e_v, e_c, m, v_g = _case()
    eps = R.rpa_epsilon(e_v, e_c, np.zeros_like(m), v_g, OMEGA)
    assert np.array_equal(eps, np.eye(len(v_g)))
    assert np.allclose(R.screened_w(eps, v_g), np.diag(v_g), rtol=0, atol=1e-15)


def test_one_transition_one_plane_wave_by_hand():
    # eps = 1 + 2 kappa v |M|^2 / (E_c - E_v), w = v / eps
    m = np.array([[[[0.3 - 0.4j]]]])            # |M|^2 = 0.25
    e_v, e_c = np.array([[-1.0]]), np.array([[2.0]])   # gap 3 eV
    v = np.array([2.0])
    kap = kappa(1, OMEGA)
    eps = 1.0 + 2.0 * kap * 2.0 * 0.25 / 3.0
    assert np.isclose(R.rpa_epsilon(e_v, e_c, m, v, OMEGA)[0, 0], eps, rtol=1e-14)
    assert np.isclose(R.screened_w(R.rpa_epsilon(e_v, e_c, m, v, OMEGA), v)[0, 0], 2.0 / eps,
                      rtol=1e-14)


def test_one_transition_two_plane_waves_by_hand():
    # X = conj(m) m^T / gap; eps = I + 2 kappa X diag(v); explicit 2 x 2 inverse
    m0, m1 = 0.5 + 0.5j, -0.2 + 0.1j
    m = np.array([m0, m1]).reshape(1, 1, 1, 2)
    e_v, e_c = np.array([[-0.5]]), np.array([[1.5]])
    v = np.array([1.5, 0.8])
    s = 2.0 * kappa(1, OMEGA) / 2.0               # 2 kappa / gap
    a = 1 + s * np.conj(m0) * m0 * v[0]
    b = s * np.conj(m0) * m1 * v[1]
    c = s * np.conj(m1) * m0 * v[0]
    d = 1 + s * np.conj(m1) * m1 * v[1]
    eps = R.rpa_epsilon(e_v, e_c, m, v, OMEGA)
    assert np.allclose(eps, [[a, b], [c, d]], rtol=1e-14, atol=0)
    det = a * d - b * c
    inv = np.array([[d, -b], [-c, a]]) / det
    assert np.allclose(R.screened_w(eps, v), v[:, None] * inv, rtol=1e-13, atol=0)


def test_sherman_morrison_one_transition():
    rng = np.random.default_rng(5)
    ng = 7
    m = (rng.standard_normal(ng) + 1j * rng.standard_normal(ng)).reshape(1, 1, 1, ng)
    e_v, e_c = np.array([[-2.0]]), np.array([[0.7]])
    v = rng.uniform(0.3, 2.0, ng)
    s = 2.0 * kappa(1, OMEGA) / 2.7
    u = np.conj(m.reshape(-1))                   # w = V - s V u u^H V / (1 + s u^H V u)
    V = np.diag(v)
    w_ref = V - s * np.outer(V @ u, np.conj(u) @ V) / (1.0 + s * np.real(np.conj(u) @ V @ u))
    w = R.screened_w(R.rpa_epsilon(e_v, e_c, m, v, OMEGA), v)
    assert np.allclose(w, w_ref, rtol=1e-12, atol=1e-14)


def test_w_is_the_inverse_of_v_inverse_plus_x():
    # v eps^-1 = v (I + X' v)^-1 = (v^-1 + X')^-1 with X' = 2 kappa X Hermitian PSD:
    # w is Hermitian, positive definite and below v (Loewner order)
    e_v, e_c, m, v_g = _case(seed=11, nk=3, nv=2, nc=4, ng=9)
    eps = R.rpa_epsilon(e_v, e_c, m, v_g, OMEGA)
    w = R.screened_w(eps, v_g)
    x = 2.0 * kappa(3, OMEGA) * R.rpa_sum(e_v, e_c, m)
    assert np.allclose(x, x.conj().T, rtol=0, atol=1e-14)
    w_ref = np.linalg.inv(np.diag(1.0 / v_g) + x)
    assert np.allclose(w, w_ref, rtol=1e-11, atol=1e-13)
    assert np.abs(w - w.conj().T).max() < 1e-12
    assert np.linalg.eigvalsh((w + w.conj().T) / 2).min() > 0
    assert np.linalg.eigvalsh(np.diag(v_g) - (w + w.conj().T) / 2).min() > -1e-12
    # the screening strictly lowers v along any direction that X sees
    assert np.trace(np.diag(v_g) - w).real > 0
