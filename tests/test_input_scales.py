"""The synthetic inputs keep A-B and A+B positive definite, which the
half-size reduction (Eq. auxham) and the Davidson product form need: the
smallest eigenvalue of each stays at least 0.3 eV above zero for the
optical-limit workload and for the 20 x 20-band, NG = 500 recipe of the
large molecular-crystal-like case on a 2x2x2 grid (its W^rr norm grows with
the grid no faster than this, the random part of the pair blocks averaging
out over more k points)."""
import dataclasses

import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O


@pytest.mark.parametrize("name,grid", [("c2", None), ("c5", 2)], ids=["c2", "c5-recipe-2x2x2"])
def test_reduction_stays_positive_definite(name, grid):
    cfg = bi.CONFIGS[name]
    if grid is not None:
        cfg = dataclasses.replace(cfg, name=f"{name}-grid{grid}", grid=grid, q_abs=(0.0,))
    p = bi.make_problem(cfg)
    A, B = O.build_A_B(p)
    assert np.linalg.eigvalsh(A - B).min() > 0.3
    assert np.linalg.eigvalsh(A + B).min() > 0.3
