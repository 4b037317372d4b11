"""Split-precision tensor-core build against the CPU oracle through the C ABI (GPU).

Tolerances: A and B within 1e-6 relative Frobenius, exciton energies within
1 meV, eps_M within 1e-3 relative at its peaks (BF16x6).  BF16x3 (two pieces,
three products) is the flagged lower-precision mode: 1e-4."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O
from test_gpu_fp64 import EDGE_SHAPES, _cluster_sums, _solve_gpu, gpu_build, problem, rel_fro

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
    assert m.mixed_available(), "the library must serve the BF16x6 tensor-core path"
    return m


def peaks(eps_im, frac=0.1):
    m = eps_im.max()
    idx = [i for i in range(1, len(eps_im) - 1)
           if eps_im[i] >= eps_im[i - 1] and eps_im[i] >= eps_im[i + 1] and eps_im[i] > frac * m]
    return np.array(idx)


# long K (NG > 192): the tensor-core tiles accumulate K in segments of <= 8
# steps summed in the epilogue; NG = 300 -> 3 segments, NG = 500 -> 4
LONG_K = [(2, 2, 3, 300), (2, 4, 4, 500)]


@pytest.mark.parametrize("name", LONG_K, ids=str)
def test_build_bf16x6_long_k(bse, name):
    p = problem(name)
    A_ref, B_ref = O.build_A_B(p)
    d = gpu_build(bse, p, precision=bse.BSE_PREC_BF16X6)
    n = p["nk"] * p["nv"] * p["nc"]
    ea = rel_fro(bse.matrix_to_numpy(d["A"], n), A_ref)
    eb = rel_fro(bse.matrix_to_numpy(d["B"], n), B_ref)
    print(f"\nlong K {name}: A {ea:.2e} B {eb:.2e}")
    assert ea < 1e-6 and eb < 1e-6, (ea, eb)


@pytest.mark.parametrize("name", ["c1", "c2"] + EDGE_SHAPES, ids=str)
def test_build_bf16x6_parity(bse, name):
    p = problem(name)
    A_ref, B_ref = O.build_A_B(p)
    d = gpu_build(bse, p, precision=bse.BSE_PREC_BF16X6)
    n = p["nk"] * p["nv"] * p["nc"]
    A = bse.matrix_to_numpy(d["A"], n)
    B = bse.matrix_to_numpy(d["B"], n)
    ea, eb = rel_fro(A, A_ref), rel_fro(B, B_ref)
    assert ea < 1e-6 and eb < 1e-6, (ea, eb)


@pytest.mark.parametrize("name", ["c1", "c2"], ids=str)
def test_build_bf16x3_parity(bse, name):
    p = problem(name)
    A_ref, B_ref = O.build_A_B(p)
    d = gpu_build(bse, p, precision=bse.BSE_PREC_BF16X3)
    n = p["nk"] * p["nv"] * p["nc"]
    assert rel_fro(bse.matrix_to_numpy(d["A"], n), A_ref) < 1e-4
    assert rel_fro(bse.matrix_to_numpy(d["B"], n), B_ref) < 1e-4


@pytest.mark.parametrize("name", ["c1", "c2"], ids=str)
@pytest.mark.parametrize("coupling", [True, False], ids=["full", "tda"])
def test_mixed_spectrum_within_1meV(bse, name, coupling):
    p = problem(name)
    n = p["nk"] * p["nv"] * p["nc"]
    A, B = O.build_A_B(p, coupling=coupling)
    e_ref, osc_ref, eps_ref = O.spectrum(A, B, p, coupling=coupling)
    d = gpu_build(bse, p, precision=bse.BSE_PREC_BF16X6, coupling=coupling)
    e, osc, eps = _solve_gpu(bse, d, n, p, coupling)
    assert np.abs(e - np.sort(e_ref)).max() < 1e-3          # 1 meV
    pk = peaks(eps_ref.imag)
    assert len(pk) > 0
    rel = np.abs(eps[pk] - eps_ref[pk]) / np.abs(eps_ref[pk])
    assert rel.max() < 1e-3


@pytest.mark.parametrize("gx,gc", [(0, 1), (1, 0), (0, 0)], ids=["triplet", "RPA", "IP"])
def test_mixed_spin_factors(bse, gx, gc):
    p = problem("c1")
    A_ref, B_ref = O.build_A_B(p, gamma_x=gx, gamma_c=gc)
    d = gpu_build(bse, p, precision=bse.BSE_PREC_BF16X6, gamma_x=gx, gamma_c=gc)
    n = p["nk"] * p["nv"] * p["nc"]
    assert rel_fro(bse.matrix_to_numpy(d["A"], n), A_ref) < 1e-6
    B = bse.matrix_to_numpy(d["B"], n)
    if np.linalg.norm(B_ref) > 0:
        assert rel_fro(B, B_ref) < 1e-6
    else:
        assert np.abs(B).max() == 0.0


def test_mixed_tda_leaves_B(bse):
    p = problem((2, 2, 3, 15))
    n = p["nk"] * p["nv"] * p["nc"]
    A_ref, _ = O.build_A_B(p, coupling=False)
    d = gpu_build(bse, p, precision=bse.BSE_PREC_BF16X6, coupling=False, ld=n + 3)
    assert rel_fro(bse.matrix_to_numpy(d["A"], n), A_ref) < 1e-6
    assert (d["B"].cpu().numpy() == complex(7.0, -3.0)).all()
    assert (d["A"][:, n:].cpu().numpy() == 0).all()
