"""The oracle's per-block build (used for sampled checks of full-size GPU
builds) and the device-side input generator, on the CPU.

block_A_B restates Eqs. vrrofM, wrrm, wrabar, diagonalblock and
couplingblock for one (k, k') block; it must reproduce every block of the
full build_A_B (itself pinned by closed forms and brute force), reduce to
the independent-particle diagonal with W = v = 0, and give Hermitian A and
B across mirrored blocks.  make_problem_torch must impose symmetries S1-S4
like make_problem."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O

UNEVEN = bi.BSEConfig("uneven", grid=2, nv=2, nc=3, ng=15, w_scale=0.2)


def _blocks_match(p, tol=1e-12):
    A, B = O.build_A_B(p)
    nk, nv, nc = p["nk"], p["nv"], p["nc"]
    s = nv * nc
    scale = max(np.abs(A).max(), np.abs(B).max())
    for k in range(nk):
        for kp in range(nk):
            a, b = O.block_A_B(bi.block_inputs(p, k, kp))
            assert np.abs(a - A[k * s:(k + 1) * s, kp * s:(kp + 1) * s]).max() < tol * scale
            assert np.abs(b - B[k * s:(k + 1) * s, kp * s:(kp + 1) * s]).max() < tol * scale


@pytest.mark.parametrize("cfg", ["c1", UNEVEN], ids=["c1", "uneven"])
def test_blocks_equal_full_build(cfg):
    _blocks_match(bi.make_problem(cfg))


def test_block_independent_particle_limit():
    p = bi.scaled(bi.make_problem(UNEVEN), w=0.0, v_bar=0.0)
    e = O.transition_energies(p["e_v"], p["e_c"]).reshape(p["nk"], -1)
    for k, kp in [(0, 0), (3, 3), (1, 5), (6, 2)]:
        a, b = O.block_A_B(bi.block_inputs(p, k, kp))
        ref = np.diag(e[k]) if k == kp else np.zeros_like(a)
        assert np.array_equal(a, ref) and not b.any()


def test_block_hermitian_across_mirror():
    p = bi.make_problem(UNEVEN)
    for k, kp in [(0, 1), (2, 7), (5, 5)]:
        a, b = O.block_A_B(bi.block_inputs(p, k, kp))
        at, bt = O.block_A_B(bi.block_inputs(p, kp, k))
        assert np.abs(a - at.conj().T).max() < 1e-13 * np.abs(a).max()
        assert np.abs(b - bt.conj().T).max() < 1e-13 * np.abs(b).max()


def _numpy_problem(pt):
    out = {}
    for k, v in pt.items():
        out[k] = v.numpy() if hasattr(v, "numpy") else v
    return out


def test_device_generator_symmetries_and_blocks():
    torch = pytest.importorskip("torch")
    cfg = bi.BSEConfig("small-torch", grid=2, nv=2, nc=3, ng=27, q_abs=(0.3,), w_scale=0.2)
    pt = bi.make_problem_torch(cfg, device="cpu")
    p = _numpy_problem(pt)
    nk, ng = p["nk"], p["ng"]
    assert p["m_vv"].shape == (nk, nk, 2, 2, ng) and p["n_vc"].shape == (nk, nk, 2, 3, ng)
    # S1: W(q) Hermitian, positive strictly dominant diagonal
    for q in range(nk):
        w = p["w"][q]
        assert np.array_equal(w, w.conj().T)
        off = np.abs(w).sum(1) - np.abs(np.diag(w))
        assert (np.diag(w).real > off).all()
    # S2: W(-q) = conj(W(q))
    _, _, neg = bi.pair_maps(2)
    for q in range(nk):
        assert np.array_equal(p["w"][neg[q]], np.conj(p["w"][q]))
    # S3: m[k',k,b',b] = conj(m[k,k',b,b'])
    for name in ("m_vv", "m_cc"):
        m = p[name]
        assert np.array_equal(m, np.conj(m.transpose(1, 0, 3, 2, 4)))
    # the block oracle on tensor-held inputs equals the full build on the same numbers
    _blocks_match(p)
    A, _ = O.build_A_B(p)
    assert np.abs(A - A.conj().T).max() < 1e-13 * np.abs(A).max()
