"""The RPA screening oracle (oracle/rpa_oracle.py) against its pins (CPU):
closed forms worked by hand and identities the definition must satisfy; and
plausible mistakes planted in a copy of the oracle, each caught by a pin."""
import os
import types

import numpy as np
import pytest

from oracle import rpa_oracle
from oracle.bse_oracle import kappa

OMEGA = 270.0
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "rpa_oracle.py")


def _case(seed=3, nk=2, nv=2, nc=3, ng=6):
    rng = np.random.default_rng(seed)
    e_v = rng.uniform(-3.0, 0.0, (nk, nv))
    e_c = rng.uniform(1.0, 4.0, (nk, nc))
    m = (rng.standard_normal((nk, nv, nc, ng)) + 1j * rng.standard_normal((nk, nv, nc, ng))) * 0.7
    v_g = rng.uniform(0.5, 3.0, ng)
    return e_v, e_c, m, v_g


def pin_no_transitions(R):
    e_v, e_c, m, v_g = _case()
    eps = R.rpa_epsilon(e_v, e_c, np.zeros_like(m), v_g, OMEGA)
    assert np.array_equal(eps, np.eye(len(v_g)))
    assert np.allclose(R.screened_w(eps, v_g), np.diag(v_g), rtol=0, atol=1e-15)


def pin_one_transition_one_plane_wave(R):
    # eps = 1 + 2 kappa v |M|^2 / (E_c - E_v), w = v / eps
    m = np.array([[[[0.3 - 0.4j]]]])            # |M|^2 = 0.25
    e_v, e_c = np.array([[-1.0]]), np.array([[2.0]])   # gap 3 eV
    v = np.array([2.0])
    eps = 1.0 + 2.0 * kappa(1, OMEGA) * 2.0 * 0.25 / 3.0
    got = R.rpa_epsilon(e_v, e_c, m, v, OMEGA)
    assert np.isclose(got[0, 0], eps, rtol=1e-14)
    assert np.isclose(R.screened_w(got, v)[0, 0], 2.0 / eps, rtol=1e-14)


def pin_one_transition_two_plane_waves(R):
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
    inv = np.array([[d, -b], [-c, a]]) / (a * d - b * c)
    assert np.allclose(R.screened_w(eps, v), v[:, None] * inv, rtol=1e-13, atol=0)


def pin_sherman_morrison(R):
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


def pin_w_is_inverse_of_v_inverse_plus_x(R):
    # v eps^-1 = v (I + X' v)^-1 = (v^-1 + X')^-1 with X' = 2 kappa X Hermitian PSD
    # (X' restated here from its definition, not taken from the oracle):
    # w is Hermitian, positive definite and below v (Loewner order)
    e_v, e_c, m, v_g = _case(seed=11, nk=3, nv=2, nc=4, ng=9)
    w = R.screened_w(R.rpa_epsilon(e_v, e_c, m, v_g, OMEGA), v_g)
    de = e_c[:, None, :] - e_v[:, :, None]                      # [k, v, c]
    mm = (m / np.sqrt(de)[..., None]).reshape(-1, m.shape[-1])
    x = 2.0 * kappa(3, OMEGA) * (np.conj(mm).T @ mm)
    w_ref = np.linalg.inv(np.diag(1.0 / v_g) + x)
    assert np.allclose(w, w_ref, rtol=1e-11, atol=1e-13)
    assert np.abs(w - w.conj().T).max() < 1e-12
    assert np.linalg.eigvalsh((w + w.conj().T) / 2).min() > 0
    assert np.linalg.eigvalsh(np.diag(v_g) - (w + w.conj().T) / 2).min() > -1e-12


PINS = [pin_no_transitions, pin_one_transition_one_plane_wave, pin_one_transition_two_plane_waves,
        pin_sherman_morrison, pin_w_is_inverse_of_v_inverse_plus_x]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(rpa_oracle)


MUTANTS = {
    "no_factor_2": ("+ 2.0 * kappa(nk", "+ 1.0 * kappa(nk"),
    "screening_sign": ("+ 2.0 * kappa(nk", "- 2.0 * kappa(nk"),
    "conj_on_g_prime": ("np.outer(np.conj(m[k, v, c]), m[k, v, c])",
                        "np.outer(m[k, v, c], np.conj(m[k, v, c]))"),
    "v_on_g": ("x * v_g[None, :]", "x * v_g[:, None]"),
    "gap_sign": ("de = e_c_kq[k, c] - e_v[k, v]", "de = e_v[k, v] - e_c_kq[k, c]"),
    "w_v_on_the_right": ("v_g[:, None] * np.linalg.inv(eps)", "np.linalg.inv(eps) * v_g[None, :]"),
    "kappa_no_nk": ("kappa(nk, omega_cell)", "kappa(1, omega_cell)"),
}


def _mutant(old, new):
    src = open(SRC).read().replace("from .bse_oracle import kappa",
                                   "from oracle.bse_oracle import kappa")
    assert src.count(old) >= 1, f"mutation anchor not found: {old}"
    mod = types.ModuleType("rpa_oracle_mutant")
    exec(compile(src.replace(old, new), "rpa_oracle_mutant", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    mod = _mutant(*MUTANTS[name])
    caught = []
    for pin in PINS:
        try:
            pin(mod)
        except Exception:      # AssertionError or a numerical failure
            caught.append(pin.__name__)
    assert caught, f"no pin caught mutant {name}"
