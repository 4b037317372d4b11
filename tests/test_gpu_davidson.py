"""Lowest excitons by block Davidson against the oracle's dense solve (GPU).

The Davidson iteration converges to the lowest eigenpairs of the product form
(A-B)(A+B)(X+Y) = E^2 (X+Y); the oracle reaches the same E by the dense
square-root reduction (Eq. auxham) and a full eigendecomposition."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O
from test_gpu_fp64 import gpu_build, problem

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


def _run(bse, d, n, nev, coupling=True, tol=1e-6, max_iter=200, precond=0, mlp=None,
         matvec_precision=0):
    import torch
    E = torch.empty(nev, dtype=torch.float64, device="cuda")
    X = torch.empty((nev, n), dtype=torch.complex128, device="cuda")
    it = bse.bse_lowest_excitons(n, d["A"], d["B"] if coupling else None, nev, E, X,
                                 tol_ev=tol, max_iter=max_iter, precond=precond, mlp=mlp,
                                 matvec_precision=matvec_precision)
    torch.cuda.synchronize()
    return E.cpu().numpy(), X.cpu().numpy().T, it


@pytest.mark.parametrize("name,nev", [("c1", 8), ("c2", 16), ((3, 2, 3, 27), 10)], ids=str)
@pytest.mark.parametrize("coupling", [True, False], ids=["full", "tda"])
def test_davidson_matches_dense(bse, name, nev, coupling):
    p = problem(name)
    n = p["nk"] * p["nv"] * p["nc"]
    A, B = O.build_A_B(p, coupling=coupling)
    if coupling:
        e_ref, _ = O.solve_full(A, B)
    else:
        e_ref = np.linalg.eigvalsh(A)
    d = gpu_build(bse, p, coupling=coupling)
    e, xpy, it = _run(bse, d, n, nev, coupling)
    assert np.abs(e - np.sort(e_ref)[:nev]).max() < 1e-8
    # the returned X+Y satisfy the product form and the normalisation
    Bm = B if coupling else np.zeros_like(A)
    xmy = ((A + Bm) @ xpy) / e[None, :]
    assert np.allclose((A - Bm) @ xmy, xpy * e[None, :], atol=1e-5)
    assert np.allclose(np.diag(xpy.conj().T @ xmy).real, 1.0, atol=1e-8)
    assert 1 <= it < 200
    print(f" [{name} nev={nev} {'full' if coupling else 'tda'}: {it} iterations]", end="")


def test_davidson_no_convergence_is_reported(bse):
    p = problem("c2")
    n = p["nk"] * p["nv"] * p["nc"]
    d = gpu_build(bse, p)
    with pytest.raises(bse.BSEError) as ei:
        _run(bse, d, n, 16, tol=1e-12, max_iter=2)
    assert ei.value.status == bse.BSE_ERR_NO_CONV


def test_davidson_argument_errors(bse):
    import torch
    p = problem("c1")
    n = p["nk"] * p["nv"] * p["nc"]
    d = gpu_build(bse, p)
    E = torch.empty(4, dtype=torch.float64, device="cuda")
    for kw, status in [(dict(nev=0), bse.BSE_ERR_ARG), (dict(nev=n + 1), bse.BSE_ERR_ARG),
                       (dict(nev=4, precond=1), bse.BSE_ERR_ARG)]:
        with pytest.raises(bse.BSEError) as ei:
            bse.bse_lowest_excitons(n, d["A"], d["B"], kw.pop("nev"), E, None, **kw)
        assert ei.value.status == status


@pytest.mark.parametrize("name,nev", [("c2", 16), ((3, 2, 3, 27), 10)], ids=str)
@pytest.mark.parametrize("coupling", [True, False], ids=["full", "tda"])
def test_davidson_tensor_core_matvecs(bse, name, nev, coupling):
    """Matvecs on the tensor cores (A, B split into BF16 pieces once): the
    energies stay within 1e-5 eV of the dense FP64 solve (the matvec error is
    ~1e-7 of |A|, far inside the 1 meV bar) at a residual tolerance of 1e-5."""
    p = problem(name)
    n = p["nk"] * p["nv"] * p["nc"]
    A, B = O.build_A_B(p, coupling=coupling)
    e_ref = O.solve_full(A, B)[0] if coupling else np.linalg.eigvalsh(A)
    d = gpu_build(bse, p, coupling=coupling)
    e, xpy, it = _run(bse, d, n, nev, coupling, tol=1e-5, matvec_precision=bse.BSE_PREC_BF16X6)
    assert np.abs(e - np.sort(e_ref)[:nev]).max() < 1e-5
    assert 1 <= it < 200
    print(f" [{name} nev={nev} {'full' if coupling else 'tda'} TC matvecs: {it} iterations]", end="")


def test_davidson_core_levels_tensor_core_matvecs(bse):
    """Core-level window (2 levels near -400 eV x 20 conduction bands): the
    transition energies on A's diagonal are 400 eV while the interaction is
    about 100 eV.  The tensor-core matvecs apply the diagonal in FP64, so the
    energies still agree with the dense FP64 solve far inside 1 meV."""
    cfg = bi.BSEConfig("core", grid=2, nv=2, nc=20, ng=59, w_scale=0.05,
                       e_v_range=(-400.5, -399.5), m_decay=0.05)
    p = bi.make_problem(cfg)
    n = p["nk"] * p["nv"] * p["nc"]
    A, B = O.build_A_B(p)
    e_ref = np.sort(O.solve_full(A, B)[0])
    d = gpu_build(bse, p)
    nev = 12
    e, xpy, it = _run(bse, d, n, nev, tol=1e-5, matvec_precision=bse.BSE_PREC_BF16X6)
    assert e_ref[0] > 399.0
    assert np.abs(e - e_ref[:nev]).max() < 1e-5
    assert 1 <= it < 200
    print(f" [core levels nev={nev} TC matvecs: {it} iterations]", end="")


def test_exciton_bands_warm_start(bse):
    """Exciton dispersion over a line of Q (a smooth family: only v(G+Q)
    changes): every Q's lowest energies match the oracle's dense solve from a
    cold or a warm start (bse_lowest_excitons_from, seeded with the previous
    Q's X+Y), and the warm starts need fewer iterations."""
    cfg = bi.BSEConfig("band", grid=4, nv=4, nc=4, ng=59, q_abs=(0.10, 0.12, 0.14, 0.16),
                       w_scale=0.25)
    nev = 12
    probs = [bi.make_problem(cfg, q_index=q, draws_of=0) for q in range(4)]
    refs = [np.sort(O.solve_full(*O.build_A_B(p))[0])[:nev] for p in probs]
    ds = [gpu_build(bse, p) for p in probs]
    n = probs[0]["nk"] * probs[0]["nv"] * probs[0]["nc"]
    items = [(n, d["A"], d["B"]) for d in ds]
    e_cold, it_cold = bse.exciton_bands(items, nev, tol_ev=1e-6, warm=False)
    e_warm, it_warm = bse.exciton_bands(items, nev, tol_ev=1e-6, warm=True)
    for q in range(4):
        assert np.abs(e_cold[q] - refs[q]).max() < 1e-8
        assert np.abs(e_warm[q] - refs[q]).max() < 1e-8
    assert it_warm[0] == it_cold[0]
    assert all(w < c for w, c in zip(it_warm[1:], it_cold[1:])), (it_warm, it_cold)
    # the dispersion itself: the lowest exciton moves with Q
    assert np.abs(refs[3][0] - refs[0][0]) > 1e-6
    print(f" [iterations cold {it_cold}, warm {it_warm}]", end="")
