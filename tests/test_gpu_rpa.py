"""Static RPA screening on the GPU (bse_rpa_screening) against the oracle
(oracle/rpa_oracle.py), FP64 (GPU)."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import rpa_oracle as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bse():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_05575_gb300 import build
    build.build()
    import paper_1904_05575_gb300 as m
    m.load()
    return m


def _case(seed, nk, nv, nc, ng):
    rng = np.random.default_rng(seed)
    e_v = rng.uniform(-3.0, 0.0, (nk, nv))
    e_c = rng.uniform(1.0, 4.0, (nk, nc))
    g2 = (bi.reciprocal_vectors(ng) ** 2).sum(1)
    m = (rng.standard_normal((nk, nv, nc, ng)) + 1j * rng.standard_normal((nk, nv, nc, ng)))
    m *= np.sqrt(0.5) / (1.0 + g2)
    q = np.array([0.2, 0.0, 0.0])
    v = 4.0 * np.pi / ((bi.reciprocal_vectors(ng) + q) ** 2).sum(1)
    return e_v, e_c, m, v


# shapes: small, several K ranges of the FP64 kernel (1,024) and of the tensor-core
# GEMM (512) with a ragged last range, NG past one 128-row tile, a single element
SHAPES = [(8, 2, 3, 15), (8, 4, 4, 59), (64, 4, 5, 181), (1, 1, 1, 1)]


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (2, 2e-6)], ids=["fp64", "bf16x6"])
@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_rpa_screening_matches_oracle(bse, shape, prec, tol):
    import torch
    nk, nv, nc, ng = shape
    e_v, e_c, m, v = _case(7, nk, nv, nc, ng)
    omega = bi.OMEGA_CELL
    eps_ref = R.rpa_epsilon(e_v, e_c, m, v, omega)
    w_ref = R.screened_w(eps_ref, v)
    t = {k: torch.as_tensor(x).cuda() for k, x in (("e_v", e_v), ("e_c", e_c), ("m", m), ("v", v))}
    w = torch.empty((ng, ng), dtype=torch.complex128, device="cuda")
    bse.bse_rpa_screening(t["e_v"], t["e_c"], t["m"], t["v"], omega, w, precision=prec)
    torch.cuda.synchronize()
    err = np.linalg.norm(w.cpu().numpy() - w_ref) / np.linalg.norm(w_ref)
    assert err < tol, err
    # the screening weakens the bare potential: w - v is the (negative) correction
    corr_ref = w_ref - np.diag(v)
    err_c = np.linalg.norm(w.cpu().numpy() - np.diag(v) - corr_ref) / np.linalg.norm(corr_ref)
    assert err_c < (1e-10 if prec == 0 else 1e-5), err_c


def test_rpa_screening_rejects_a_negative_gap(bse):
    import torch
    e_v, e_c, m, v = _case(3, 2, 1, 1, 5)
    e_c[1, 0] = e_v[1, 0] - 0.1
    t = [torch.as_tensor(x).cuda() for x in (e_v, e_c, m, v)]
    w = torch.empty((5, 5), dtype=torch.complex128, device="cuda")
    with pytest.raises(bse.BSEError) as ei:
        bse.bse_rpa_screening(*t, bi.OMEGA_CELL, w)
    assert ei.value.status == bse.BSE_ERR_ARG
