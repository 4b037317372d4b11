"""k-row slabs: A and B built a slab of k rows at a time (GPU).

The exchange (Eq. vrrofM) and both direct terms (Eqs. wrrm, wrabar) are sums
over independent (k, k') blocks, so the rows (k v c) of A and B with k in a
slab need only the slab's rows of m_vv and m_cc (n_vc stays whole: W^ra of
row k reads n_vc[k'][k]).  Each test builds a problem slab by slab into one
A and B (slab arrays are row slices of the whole device arrays) and compares
the union with the oracle's whole A and B; a single slab must leave every
other row untouched.  Paths: FP64, the fused tensor-core direct term
(Nv = Nc = 2), the two-launch form with CUDA-core stage 2 (an uneven window,
W applied to the valence side; the core-level window with its skinny W^rr
and 40 x 40 W^ra blocks), and the tensor-core stage 2 (8 x 8 bands).
"""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O

pytestmark = pytest.mark.gpu

FP64_TOL, MIXED_TOL = 1e-12, 1e-6   # relative Frobenius, as in the other parity tests


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


SHAPES = {
    # 2x2x2 grid, 2x2 bands: fused direct term
    "c1": bi.CONFIGS["c1"],
    # uneven window: W applied to the 4 (v, v') rows, the 9 (c, c') rows contracted after
    "v2c3": bi.BSEConfig("slab-v2c3", grid=2, nv=2, nc=3, ng=59, w_scale=0.1),
    # 8 x 8 bands: 64-row pair blocks, stage 2 on the tensor cores
    "v8c8": bi.BSEConfig("slab-v8c8", grid=2, nv=8, nc=8, ng=59, w_scale=0.05),
    # the core-level window (2 x 20 bands): 4 T rows against 400 X rows (one
    # thread per X row) and 40 x 40 W^ra blocks (one 40 x 40 tile per pair)
    "v2c20": bi.BSEConfig("slab-v2c20", grid=2, nv=2, nc=20, ng=59, w_scale=0.05,
                          e_v_range=(-400.5, -399.5), m_decay=0.05),
    # 4 T rows against 64 X rows: a block of 128 X rows spans three pair blocks
    "v2c8": bi.BSEConfig("slab-v2c8", grid=2, nv=2, nc=8, ng=59, w_scale=0.1),
    # 4 T rows against 36 (c, c') rows, and 4 (c, c') T rows against 16 (v, v')
    # X rows (W applied to the conduction side): up to nine pair blocks per
    # block of 128 X rows
    "v2c6": bi.BSEConfig("slab-v2c6", grid=2, nv=2, nc=6, ng=59, w_scale=0.1),
    "v4c2": bi.BSEConfig("slab-v4c2", grid=2, nv=4, nc=2, ng=59, w_scale=0.1),
}


@pytest.fixture(scope="module")
def cases():
    out = {}
    for name, cfg in SHAPES.items():
        p = bi.make_problem(cfg)
        out[name] = (p, O.build_A_B(p))
    return out


def _rel(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


def _rel_interaction(p, A, A_ref):
    """Error of A without its E^ip diagonal (which dominates A's norm when the
    transition energies are hundreds of eV, as for core levels)."""
    D = np.diag(O.transition_energies(p["e_v"], p["e_c"]).astype(np.complex128))
    return _rel(A - D, A_ref - D)


def _slab_view(d, kb, kn):
    """The problem dict with m_vv and m_cc cut to rows [kb, kb + kn) (views)."""
    s = dict(d)
    s["m_vv"] = d["m_vv"][kb:kb + kn]
    s["m_cc"] = d["m_cc"][kb:kb + kn]
    return s


def _build_slabs(bse, d, slabs, prec, fused=True, one_call=False):
    import torch
    structs = [bse.make_problem_struct(_slab_view(d, kb, kn), k_begin=kb, k_count=kn)
               for kb, kn in slabs]
    if prec == bse.BSE_PREC_FP64 or one_call:
        if one_call:
            bse.bse_build_kernel(structs, prec)
        else:
            for st in structs:
                bse.bse_build_kernel([st], prec)
    else:
        for st in structs:
            plan = bse.Plan([st], precision=prec, fused=fused)
            plan.execute()
            plan.status()
            plan.close()
    torch.cuda.synchronize()


PATHS = [("c1", 0, True), ("c1", 2, True), ("c1", 2, False), ("v2c3", 0, True),
         ("v2c3", 2, True), ("v8c8", 0, True), ("v8c8", 2, True), ("v2c20", 0, True),
         ("v2c20", 2, True), ("v2c8", 2, True), ("v2c6", 2, True), ("v4c2", 2, True)]


@pytest.mark.parametrize("shape,prec,fused", PATHS,
                         ids=[f"{s}-{'fp64' if p == 0 else 'bf16x6'}{'' if f else '-unfused'}"
                              for s, p, f in PATHS])
def test_slabs_cover_the_whole_problem(bse, cases, shape, prec, fused):
    p, (A_ref, B_ref) = cases[shape]
    nk = p["nk"]
    n = nk * p["nv"] * p["nc"]
    d = bse.upload_problem(p)
    # ragged slabs, one of a single k row
    slabs = [(0, 3), (3, 1), (4, nk - 4)]
    _build_slabs(bse, d, slabs, prec, fused)
    tol = FP64_TOL if prec == 0 else MIXED_TOL
    A = bse.matrix_to_numpy(d["A"], n)
    ea, ei = _rel(A, A_ref), _rel_interaction(p, A, A_ref)
    eb = _rel(bse.matrix_to_numpy(d["B"], n), B_ref)
    assert ea < tol and ei < tol and eb < tol, (ea, ei, eb)


@pytest.mark.parametrize("prec", [0, 2], ids=["fp64", "bf16x6"])
def test_slabs_in_one_call(bse, cases, prec):
    """Two slabs of one problem as two problems of one batched call."""
    p, (A_ref, B_ref) = cases["c1"]
    n = p["nk"] * p["nv"] * p["nc"]
    d = bse.upload_problem(p)
    _build_slabs(bse, d, [(0, 5), (5, 3)], prec, one_call=True)
    tol = FP64_TOL if prec == 0 else MIXED_TOL
    assert _rel(bse.matrix_to_numpy(d["A"], n), A_ref) < tol
    assert _rel(bse.matrix_to_numpy(d["B"], n), B_ref) < tol


@pytest.mark.parametrize("shape,prec", [("c1", 0), ("c1", 2), ("v8c8", 2)],
                         ids=["c1-fp64", "c1-bf16x6", "v8c8-bf16x6"])
def test_one_slab_leaves_other_rows(bse, cases, shape, prec):
    import torch
    p, (A_ref, B_ref) = cases[shape]
    s = p["nv"] * p["nc"]
    n = p["nk"] * s
    d = bse.upload_problem(p)
    d["A"].fill_(complex(123.0, -45.0))
    d["B"].fill_(complex(-9.0, 8.0))
    kb, kn = 2, 3
    _build_slabs(bse, d, [(kb, kn)], prec)
    A, B = bse.matrix_to_numpy(d["A"], n), bse.matrix_to_numpy(d["B"], n)
    rows = np.zeros(n, bool)
    rows[kb * s:(kb + kn) * s] = True
    assert (A[~rows] == complex(123.0, -45.0)).all()
    assert (B[~rows] == complex(-9.0, 8.0)).all()
    tol = FP64_TOL if prec == 0 else MIXED_TOL
    assert _rel(A[rows], A_ref[rows]) < tol
    assert _rel(B[rows], B_ref[rows]) < tol
    torch.cuda.synchronize()


def test_static_fp64_slab(bse, cases):
    """The allocation-free FP64 entry point builds a slab like the allocating one."""
    import torch
    p, (A_ref, B_ref) = cases["v2c3"]
    n = p["nk"] * p["nv"] * p["nc"]
    d = bse.upload_problem(p)
    for kb, kn in [(0, 6), (6, 2)]:
        bse.bse_build_kernel_fp64_static(
            bse.make_problem_struct(_slab_view(d, kb, kn), k_begin=kb, k_count=kn))
    torch.cuda.synchronize()
    assert _rel(bse.matrix_to_numpy(d["A"], n), A_ref) < FP64_TOL
    assert _rel(bse.matrix_to_numpy(d["B"], n), B_ref) < FP64_TOL


def test_slab_shape_checks(bse, cases):
    p, _ = cases["c1"]
    d = bse.upload_problem(p)
    with pytest.raises(ValueError):   # m_vv, m_cc still whole
        bse.make_problem_struct(d, k_begin=0, k_count=3)
    with pytest.raises(ValueError):   # past nk
        bse.make_problem_struct(_slab_view(d, 6, 3), k_begin=6, k_count=3)
