"""The build entry point that allocates no device memory (GPU).

bse_build_kernel_fp64_static serves callers that cannot allocate device memory
when they call the library: it keeps the direct terms' intermediate in a fixed
16 MiB array compiled into libbse.so.  Its output must match the allocating
FP64 build (bse_build_kernel with BSE_PREC_FP64) to the FP64 tolerance of the
other parity tests, on consecutive calls that share that array, and it must
refuse problems whose intermediate does not fit.  This file is collected last
so that a failure here does not hide the results of the other tests."""
import numpy as np
import pytest

import bse_inputs as bi

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12   # relative Frobenius, as in the FP64 parity tests


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


def _small(grid, nv, nc, ng, seed=3):
    cfg = bi.BSEConfig("noalloc", grid=grid, nv=nv, nc=nc, ng=ng, w_scale=0.1, n_omega=10)
    return bi.make_problem(cfg, seed=seed)


def _build_both(bse, p, coupling=True):
    """(static result, allocating result) as numpy N x N pairs (A, B)."""
    import torch
    n = p["nk"] * p["nv"] * p["nc"]
    d_ref = bse.upload_problem(p)
    bse.bse_build_kernel([bse.make_problem_struct(d_ref, coupling=coupling)], bse.BSE_PREC_FP64)
    d = bse.upload_problem(p)
    # garbage in the outputs: the static path must overwrite A (and B) completely
    d["A"].fill_(complex(123.0, -45.0))
    d["B"].fill_(complex(-9.0, 8.0))
    bse.bse_build_kernel_fp64_static(bse.make_problem_struct(d, coupling=coupling))
    torch.cuda.synchronize()
    out = [bse.matrix_to_numpy(d["A"], n), bse.matrix_to_numpy(d["B"], n)]
    ref = [bse.matrix_to_numpy(d_ref["A"], n), bse.matrix_to_numpy(d_ref["B"], n)]
    return out, ref


def _rel(x, ref):
    return np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300)


def test_static_matches_allocating_build_on_consecutive_calls(bse):
    # call 1 and call 2 use different shapes (conduction side, then valence side
    # of the W^rr contraction), call 3 repeats call 1: the shared array keeps
    # whatever the previous call left, and that must not matter
    cases = [_small(2, 2, 2, 59), _small(1, 1, 3, 17, seed=5), _small(2, 2, 2, 59)]
    for p in cases:
        (a, b), (a_ref, b_ref) = _build_both(bse, p)
        assert _rel(a, a_ref) < FP64_TOL
        assert _rel(b, b_ref) < FP64_TOL


def test_static_tda_leaves_b(bse):
    import torch
    p = _small(2, 2, 3, 15)
    n = p["nk"] * p["nv"] * p["nc"]
    d_ref = bse.upload_problem(p)
    bse.bse_build_kernel([bse.make_problem_struct(d_ref, coupling=False)], bse.BSE_PREC_FP64)
    d = bse.upload_problem(p)
    d["B"].fill_(complex(7.0, -3.0))
    bse.bse_build_kernel_fp64_static(bse.make_problem_struct(d, coupling=False))
    torch.cuda.synchronize()
    assert _rel(bse.matrix_to_numpy(d["A"], n), bse.matrix_to_numpy(d_ref["A"], n)) < FP64_TOL
    assert (d["B"].cpu().numpy() == complex(7.0, -3.0)).all()


def test_static_rejects_problem_beyond_fixed_scratch(bse):
    # 27 k points, 4 x 4 bands, 181 plane waves: 729 * 16 * 181 * 16 B = 33.8 MB > 16 MiB
    p = _small(3, 4, 4, 181)
    d = bse.upload_problem(p)
    with pytest.raises(bse.BSEError) as ei:
        bse.bse_build_kernel_fp64_static(bse.make_problem_struct(d))
    assert ei.value.status == bse.BSE_ERR_ARG
    assert "fixed scratch" in ei.value.message
    assert (d["A"].cpu().numpy() == 0).all()        # nothing launched
