"""Pins for the pair-element oracle (oracle/pair_oracle.py), independent of its
formulas: the matrix elements evaluated as integrals on a real-space grid of
the Bloch functions built from the same coefficients, and the orthonormality
of the bands at G = 0, q = 0; planted mistakes in a copy of the oracle are
each caught (CPU)."""
import os
import types

import numpy as np
import pytest

import bse_inputs as bi
from oracle import pair_oracle as PO

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "pair_oracle.py")
N, NV, NC, NPW, NG = 2, 2, 2, 15, 9


def _case():
    """Generic coefficients (no time-reversal relation, not orthonormal except
    at k = 0 and 1 where the bands are orthonormalised): the pins hold for
    any Bloch functions."""
    rng = np.random.default_rng(3)
    basis = bi.reciprocal_coords(NPW)
    nk = N ** 3
    c = rng.standard_normal((nk, NV + NC, NPW)) + 1j * rng.standard_normal((nk, NV + NC, NPW))
    for k in range(nk):
        q, _ = np.linalg.qr(c[k].T)
        c[k] = q.T
    return c[:, :NV], c[:, NV:], basis, bi.reciprocal_coords(NG), bi.k_grid(N)


def _real_space(cv, cc, basis, gout, kint):
    """Bloch functions on the grid of fractional coordinates of the N^3-cell
    supercell, m points per cell and direction, fine enough that no product
    of the integrands aliases (m above twice the basis radius plus the
    output radius plus one)."""
    m = 2 * int(np.abs(basis).max()) + int(np.abs(gout).max()) + 3
    x1 = np.arange(N * m) / m
    x = np.stack(np.meshgrid(x1, x1, x1, indexing="ij"), -1).reshape(-1, 3)
    def phi(c, k):
        f = basis + kint[k][None, :] / N
        return c @ np.exp(2j * np.pi * f @ x.T)
    pv = [phi(cv[k], k) for k in range(len(kint))]
    pc = [phi(cc[k], k) for k in range(len(kint))]
    return x, pv, pc


def pin_real_space(P):
    cv, cc, basis, gout, kint = _case()
    got = P.pair_elements(cv, cc, basis, gout, kint, N)
    x, pv, pc = _real_space(cv, cc, basis, gout, kint)
    npts = len(x)
    qm, qp, _ = bi.pair_maps(N)
    def integral(bra, ket, q):   # <bra| e^{-i(G+q)r} |ket> for every output G
        ph = np.exp(-2j * np.pi * (gout + q[None, :] / N) @ x.T)
        return np.einsum("ar,gr,br->abg", bra.conj(), ph, ket) / npts
    nk = len(kint)
    for k in range(nk):
        ref = integral(pc[k], pv[k], np.zeros(3))                     # [c, v, G]
        assert np.allclose(got["m_x"][k], ref.transpose(1, 0, 2), atol=1e-13), "m_x"
        for kp in range(nk):
            q = kint[qm[k, kp]]
            ref = integral(pv[kp], pv[k], q)                          # [v', v, G]
            assert np.allclose(got["m_vv"][k, kp], ref.transpose(1, 0, 2), atol=1e-13), "m_vv"
            ref = integral(pc[kp], pc[k], q)
            assert np.allclose(got["m_cc"][k, kp], ref.transpose(1, 0, 2), atol=1e-13), "m_cc"
            q = kint[qp[k, kp]]
            ref = integral(pv[k], pc[kp].conj(), q)                    # [v, c', G]
            assert np.allclose(got["n_vc"][k, kp], ref, atol=1e-13), "n_vc"


def pin_orthonormal(P):
    cv, cc, basis, gout, kint = _case()
    got = P.pair_elements(cv, cc, basis, gout, kint, N)
    g0 = int(np.where((gout == 0).all(1))[0][0])
    assert np.abs(got["m_x"][..., g0]).max() < 1e-14, "<c k|v k> = 0"
    for k in range(len(kint)):
        assert np.allclose(got["m_vv"][k, k, :, :, g0], np.eye(NV), atol=1e-14)
        assert np.allclose(got["m_cc"][k, k, :, :, g0], np.eye(NC), atol=1e-14)


PINS = [pin_real_space, pin_orthonormal]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(PO)


MUTANTS = {
    "m_conj_on_ket": ("tot += np.conj(a[i1]) * b[j]", "tot += a[i1] * np.conj(b[j])"),
    "m_no_umklapp": ("j = idx.get(tuple(int(x) for x in (g1 + G + s)))",
                     "j = idx.get(tuple(int(x) for x in (g1 + G)))"),
    "m_sign_of_G": ("j = idx.get(tuple(int(x) for x in (g1 + G + s)))",
                    "j = idx.get(tuple(int(x) for x in (g1 - G + s)))"),
    "n_no_conj_ket": ("tot += np.conj(a[i1]) * np.conj(b[j])", "tot += np.conj(a[i1]) * b[j]"),
    "n_shift_sign": ("j = idx.get(tuple(int(x) for x in (-g1 - G - s)))",
                     "j = idx.get(tuple(int(x) for x in (-g1 - G + s)))"),
    "vv_bra_ket_swapped": ("element_m(cv[kp, vp], cv[k, v], basis, gout[g], s)",
                           "element_m(cv[k, v], cv[kp, vp], basis, gout[g], s)"),
    "umklapp_sign": ("        return q_index, s\n    s = (kint[k]", "        return q_index, -s\n    s = (kint[k]"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    mod = types.ModuleType("pair_oracle_mutant")
    exec(compile(src.replace(old, new), "pair_oracle_mutant", "exec"), mod.__dict__)
    caught = []
    for pin in PINS:
        try:
            pin(mod)
        except Exception:
            caught.append(pin.__name__)
    assert caught, f"no pin caught mutant {name}"


def test_time_reversal_of_the_inputs():
    """The seeded coefficients of bse_inputs: orthonormal bands and
    phi_{n,-k} = phi_{n,k}^*, i.e. C_{n,-k}(G) = conj(C_{n,k}(-G))."""
    cv, cc, basis = bi.wavefunction_coefficients(3, NV, NC, NPW, seed=3)
    c = np.concatenate([cv, cc], 1)
    for k in range(27):
        assert np.allclose(c[k].conj() @ c[k].T, np.eye(NV + NC), atol=1e-14)
    lut = {tuple(g): i for i, g in enumerate(basis)}
    minus = np.array([lut[tuple(-g)] for g in basis])
    _, _, neg = bi.pair_maps(3)
    for c in (cv, cc):
        for k in range(27):
            assert np.allclose(c[neg[k]], np.conj(c[k][:, minus]), atol=0)
