"""Pair arrays drawn a slab of k rows at a time (bse_inputs.pair_slab_torch), on
the CPU: slabs are reproducible on their own, agree with one another where
they overlap, and together keep the symmetry S3 that makes A Hermitian
(checked through the oracle on a small shape; B comes out Hermitian too, as
the time-reversal basis of Eq. Hetr gives it)."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O

torch = pytest.importorskip("torch")

CFG = bi.BSEConfig("slab-gen", grid=2, nv=2, nc=3, ng=15, w_scale=0.1)


def test_slabs_reproducible_and_consistent():
    whole_vv, whole_cc = bi.pair_slab_torch(CFG, 0, CFG.nk, device="cpu")
    a_vv, a_cc = bi.pair_slab_torch(CFG, 2, 3, device="cpu")
    b_vv, b_cc = bi.pair_slab_torch(CFG, 2, 3, device="cpu")
    assert torch.equal(a_vv, b_vv) and torch.equal(a_cc, b_cc)
    assert torch.equal(a_vv, whole_vv[2:5]) and torch.equal(a_cc, whole_cc[2:5])


def test_slabs_keep_s3_across_slabs():
    parts = [bi.pair_slab_torch(CFG, kb, kn, device="cpu") for kb, kn in ((0, 3), (3, 1), (4, 4))]
    for i, name in enumerate(("m_vv", "m_cc")):
        x = torch.cat([p[i] for p in parts]).numpy()
        # X[k', k, b', b] = conj(X[k, k', b, b'])
        assert np.array_equal(x, np.conj(x.transpose(1, 0, 3, 2, 4))), name
        assert np.abs(x).max() > 0


def test_slab_drawn_problem_gives_hermitian_A_and_B():
    p = bi.make_problem_torch(CFG, device="cpu", k_slab=(0, CFG.nk))
    h = {k: (v.numpy() if hasattr(v, "numpy") else v) for k, v in p.items()}
    A, B = O.build_A_B(h)
    assert np.abs(A - A.conj().T).max() < 1e-12 * np.abs(A).max()
    assert np.abs(B - B.conj().T).max() < 1e-12 * np.abs(B).max()
