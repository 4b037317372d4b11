"""FP64 CUDA path against the CPU oracle through the C ABI (GPU)."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O

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


_cache = {}


def problem(name, **kw):
    key = (name, tuple(sorted(kw.items())))
    if key not in _cache:
        if name in bi.CONFIGS:
            _cache[key] = bi.make_problem(name, **kw)
        else:
            grid, nv, nc, ng = name
            cfg = bi.BSEConfig("edge", grid=grid, nv=nv, nc=nc, ng=ng, w_scale=0.1,
                               n_omega=300)
            _cache[key] = bi.make_problem(cfg, **kw)
    return _cache[key]


def gpu_build(bse, p, precision=0, gamma_x=1.0, gamma_c=1.0, coupling=True, ld=None):
    import torch
    d = bse.upload_problem(p, ld=ld)
    if not coupling:
        d["B"].fill_(complex(7.0, -3.0))      # sentinel: TDA must not touch B
    st = bse.make_problem_struct(d, gamma_x, gamma_c, coupling)
    bse.bse_build_kernel([st], precision)
    torch.cuda.synchronize()
    return d


def rel_fro(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


EDGE_SHAPES = [
    (1, 1, 3, 5),      # one k point, nv^2 < nc^2 (W applied on the valence side)
    (2, 3, 1, 17),     # nv^2 > nc^2, ragged ng
    (2, 2, 2, 1),      # a single plane wave
    (3, 2, 3, 27),     # 27 k points, N = 162 spans several 64-wide tiles
    (2, 1, 1, 59),     # N = 8
]


@pytest.mark.parametrize("name", ["c1", "c2"] + EDGE_SHAPES, ids=str)
def test_build_fp64_parity(bse, name):
    p = problem(name)
    A_ref, B_ref = O.build_A_B(p)
    d = gpu_build(bse, p)
    n = p["nk"] * p["nv"] * p["nc"]
    A = bse.matrix_to_numpy(d["A"], n)
    B = bse.matrix_to_numpy(d["B"], n)
    assert rel_fro(A, A_ref) < 1e-12
    assert rel_fro(B, B_ref) < 1e-12
    assert np.abs(A - A_ref).max() < 1e-11 * np.abs(A_ref).max()
    assert np.abs(B - B_ref).max() < 1e-11 * np.abs(B_ref).max()


@pytest.mark.parametrize("gx,gc", [(0, 1), (1, 0), (0, 0)], ids=["triplet", "RPA", "IP"])
def test_spin_factors(bse, gx, gc):
    p = problem("c1")
    A_ref, B_ref = O.build_A_B(p, gamma_x=gx, gamma_c=gc)
    d = gpu_build(bse, p, gamma_x=gx, gamma_c=gc)
    n = p["nk"] * p["nv"] * p["nc"]
    assert np.allclose(bse.matrix_to_numpy(d["A"], n), A_ref, rtol=0, atol=1e-12 * np.abs(A_ref).max())
    assert np.allclose(bse.matrix_to_numpy(d["B"], n), B_ref, rtol=0,
                       atol=1e-12 * max(np.abs(B_ref).max(), 1.0))


def test_tda_leaves_B_and_ld_padding(bse):
    p = problem((2, 2, 3, 15))
    n = p["nk"] * p["nv"] * p["nc"]
    A_ref, _ = O.build_A_B(p, coupling=False)
    d = gpu_build(bse, p, coupling=False, ld=n + 5)
    A = bse.matrix_to_numpy(d["A"], n)
    assert rel_fro(A, A_ref) < 1e-12
    # B untouched, padding rows of the column-major storage untouched
    assert (d["B"].cpu().numpy() == complex(7.0, -3.0)).all()
    assert (d["A"][:, n:].cpu().numpy() == 0).all()


def test_q_map_out_of_range_is_arg_error(bse):
    import torch
    p = dict(problem("c1"))
    qm = p["q_minus"].copy()
    qm[1, 0] = p["nk"] + 3
    p["q_minus"] = qm
    d = bse.upload_problem(p)
    st = bse.make_problem_struct(d)
    with pytest.raises(bse.BSEError) as ei:
        bse.bse_build_kernel([st], 0)
    assert ei.value.status == bse.BSE_ERR_ARG and "q_minus" in ei.value.message
    assert (d["A"].cpu().numpy() == 0).all()      # nothing launched


def _solve_gpu(bse, d, n, p, coupling=True):
    import torch
    dev = "cuda"
    S = torch.empty((n, n), dtype=torch.complex128, device=dev)
    L = torch.empty((n, n), dtype=torch.complex128, device=dev)
    bse.bse_reduce(n, d["A"], d["B"] if coupling else None, S, L)
    E = torch.empty(n, dtype=torch.float64, device=dev)
    osc = torch.empty(n, dtype=torch.float64, device=dev)
    om = torch.as_tensor(p["omega"]).to(dev)
    eps = torch.empty(len(p["omega"]), dtype=torch.complex128, device=dev)
    rho = torch.as_tensor(p["rho"]).to(dev)
    vc = p["nk"] * p["omega_cell"]
    bse.bse_spectrum(n, S, L, rho, p["c_q"], vc, om, p["delta"], E, osc, eps)
    torch.cuda.synchronize()
    return E.cpu().numpy(), osc.cpu().numpy(), eps.cpu().numpy()


def _cluster_sums(e, osc, tol=1e-6):
    """Oscillator strengths summed over degenerate clusters (|dE| < tol eV)."""
    out, cur, last = [], 0.0, None
    for ei, oi in zip(e, osc):
        if last is not None and ei - last > tol:
            out.append(cur)
            cur = 0.0
        cur += oi
        last = ei
    out.append(cur)
    return np.array(out)


@pytest.mark.parametrize("name", ["c1", "c2", (3, 2, 3, 27)], ids=str)
@pytest.mark.parametrize("coupling", [True, False], ids=["full", "tda"])
def test_reduce_spectrum_parity(bse, name, coupling):
    p = problem(name)
    n = p["nk"] * p["nv"] * p["nc"]
    A, B = O.build_A_B(p, coupling=coupling)
    e_ref, osc_ref, eps_ref = O.spectrum(A, B, p, coupling=coupling)
    d = gpu_build(bse, p, coupling=coupling)
    e, osc, eps = _solve_gpu(bse, d, n, p, coupling)
    assert np.abs(e - np.sort(e_ref)).max() < 1e-10
    order = np.argsort(e_ref)
    assert np.allclose(_cluster_sums(e, osc), _cluster_sums(e_ref[order], osc_ref[order]),
                       rtol=1e-8, atol=1e-12 * osc_ref.max())
    assert np.abs(eps - eps_ref).max() < 1e-8 * np.abs(eps_ref).max()


def test_not_positive_definite(bse):
    import torch
    p = bi.scaled(problem("c1"), w=200.0)
    n = p["nk"] * p["nv"] * p["nc"]
    A, B = O.build_A_B(p)
    assert np.linalg.eigvalsh(A - B).min() < 0
    d = gpu_build(bse, p)
    S = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    L = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    with pytest.raises(bse.BSEError) as ei:
        bse.bse_reduce(n, d["A"], d["B"], S, L)
    assert ei.value.status == bse.BSE_ERR_NOT_PD
    assert 1 <= ei.value.minor <= n
