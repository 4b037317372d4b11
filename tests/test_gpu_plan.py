"""Batched plans: several momentum transfers with uneven band windows built by
one plan, against the oracle; the plan's execute captured in a CUDA graph and
replayed; the tile-width autotuner; the fused direct term (stage-1 GEMM and
contraction in one launch) against the oracle and, bit for bit, against the
two-launch form (GPU)."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import bse_oracle as O

pytestmark = pytest.mark.gpu

# three Q along [100] with different (nv, nc) windows and one NG (a small
# version of the 16-Q finite-momentum batch)
MULTI = bi.BSEConfig("multi-q", grid=2, nv=4, nc=6, ng=59, q_abs=(0.1, 0.6, 1.1),
                     windows=((2, 2), (3, 5), (4, 6)), w_scale=0.1)


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


@pytest.fixture(scope="module")
def batch():
    probs = [bi.make_problem(MULTI, q_index=q) for q in range(3)]
    refs = [O.build_A_B(p) for p in probs]
    return probs, refs


# three Q whose windows all fit the fused direct term (Nv = Nc in {2, 4}):
# 2x2 windows put 32 pairs in a 128-row tile, and every q group ends in a
# ragged tile
SQUARE = bi.BSEConfig("multi-q-square", grid=2, nv=4, nc=4, ng=59, q_abs=(0.1, 0.6, 1.1),
                      windows=((2, 2), (4, 4), (2, 2)), w_scale=0.1)


def _rel(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


def _upload(bse, probs):
    ds = [bse.upload_problem(p) for p in probs]
    structs = [bse.make_problem_struct(d) for d in ds]
    return ds, structs


def _check(bse, probs, refs, ds, tol):
    for p, (A_ref, B_ref), d in zip(probs, refs, ds):
        n = p["nk"] * p["nv"] * p["nc"]
        assert _rel(bse.matrix_to_numpy(d["A"], n), A_ref) < tol
        assert _rel(bse.matrix_to_numpy(d["B"], n), B_ref) < tol


@pytest.mark.parametrize("prec,tol", [(2, 1e-6), (0, 1e-12)], ids=["bf16x6", "fp64"])
def test_plan_matches_oracle(bse, batch, prec, tol):
    import torch
    probs, refs = batch
    ds, structs = _upload(bse, probs)
    plan = bse.Plan(structs, precision=prec)
    for _ in range(2):                      # a plan is reusable
        for d in ds:
            d["A"].zero_()
            d["B"].zero_()
        plan.execute()
        plan.status()
        torch.cuda.synchronize()
        _check(bse, probs, refs, ds, tol)
    plan.close()


def test_plan_graph_capture_replay(bse, batch):
    import torch
    probs, refs = batch
    ds, structs = _upload(bse, probs)
    plan = bse.Plan(structs, precision=bse.BSE_PREC_BF16X6)
    stream = torch.cuda.Stream()
    plan.execute(stream)                    # eager result
    stream.synchronize()
    eager = [d["A"].clone() for d in ds] + [d["B"].clone() for d in ds]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            plan.execute(stream)
    for d in ds:
        d["A"].fill_(complex(5.0, 5.0))
        d["B"].fill_(complex(5.0, 5.0))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    plan.status()
    replayed = [d["A"] for d in ds] + [d["B"] for d in ds]
    for e, r in zip(eager, replayed):
        assert torch.equal(e, r)
    _check(bse, probs, refs, ds, 1e-6)
    plan.close()


def test_plan_autotune(bse, batch):
    import torch
    probs, refs = batch
    ds, structs = _upload(bse, probs)
    plan = bse.Plan(structs, precision=bse.BSE_PREC_BF16X6, autotune=True)
    assert plan.tile_cols in (32, 64)       # NG = 59 pads to 64: one or two tiles
    plan.execute()
    plan.status()
    torch.cuda.synchronize()
    _check(bse, probs, refs, ds, 1e-6)
    plan.close()


def test_plan_needs_one_ng(bse, batch):
    probs, _ = batch
    other = bi.make_problem(bi.BSEConfig("ng15", grid=2, nv=2, nc=2, ng=15, w_scale=0.1))
    ds, structs = _upload(bse, [probs[0], other])
    with pytest.raises(bse.BSEError) as ei:
        bse.Plan(structs, precision=bse.BSE_PREC_BF16X6)
    assert ei.value.status == bse.BSE_ERR_UNSUPPORTED
    fp64 = bse.Plan(structs, precision=bse.BSE_PREC_FP64)   # FP64 plans take any shapes
    fp64.execute()
    fp64.close()


def test_plan_with_odd_windows_is_not_fused(bse, batch):
    probs, _ = batch
    ds, structs = _upload(bse, probs)
    plan = bse.Plan(structs, precision=bse.BSE_PREC_BF16X6)
    assert not plan.fused           # 3x5 and 4x6 windows: pair blocks too tall for the epilogue
    plan.close()


@pytest.fixture(scope="module")
def square():
    probs = [bi.make_problem(SQUARE, q_index=q) for q in range(3)]
    refs = [O.build_A_B(p) for p in probs]
    return probs, refs


def _build(bse, plan, ds):
    import torch
    for d in ds:
        d["A"].fill_(complex(7.0, -7.0))
        d["B"].fill_(complex(7.0, -7.0))
    plan.execute()
    plan.status()
    torch.cuda.synchronize()
    return [d["A"].clone() for d in ds] + [d["B"].clone() for d in ds]


@pytest.mark.parametrize("prec,tol", [(2, 1e-6), (3, 1e-4)], ids=["bf16x6", "bf16x3"])
def test_fused_matches_oracle_and_two_launch_form(bse, square, prec, tol):
    import torch
    probs, refs = square
    ds, structs = _upload(bse, probs)
    fused = bse.Plan(structs, precision=prec)
    split = bse.Plan(structs, precision=prec, fused=False)
    assert fused.fused and not split.fused
    a = _build(bse, fused, ds)
    _check(bse, probs, refs, ds, tol)
    b = _build(bse, split, ds)
    for x, y in zip(a, b):
        assert torch.equal(x, y), (x - y).abs().max().item()
    fused.close()
    split.close()


@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_fused_one_call_build_is_bitwise_two_launch(bse, cfg):
    """bse_build_kernel (cached fused plan) against an explicit two-launch plan."""
    import torch
    p = bi.make_problem(cfg)
    d = bse.upload_problem(p)
    st = bse.make_problem_struct(d)
    bse.bse_build_kernel([st], bse.BSE_PREC_BF16X6)
    torch.cuda.synchronize()
    one = [d["A"].clone(), d["B"].clone()]
    split = bse.Plan([st], precision=bse.BSE_PREC_BF16X6, fused=False)
    two = _build(bse, split, [d])
    for x, y in zip(one, two):
        assert torch.equal(x, y), (x - y).abs().max().item()
    split.close()


def test_fused_graph_capture_and_autotune_leaves_outputs(bse, square):
    import torch
    probs, refs = square
    ds, structs = _upload(bse, probs)
    for d in ds:
        d["A"].fill_(complex(3.0, 1.0))
        d["B"].fill_(complex(3.0, 1.0))
    torch.cuda.synchronize()
    plan = bse.Plan(structs, precision=bse.BSE_PREC_BF16X6, autotune=True)
    assert plan.fused and plan.tile_cols in (32, 64)
    for d in ds:                     # autotuning times the fused launch with outputs off
        assert bool((d["A"] == complex(3.0, 1.0)).all()) and bool((d["B"] == complex(3.0, 1.0)).all())
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            plan.execute(stream)
    g.replay()
    torch.cuda.synchronize()
    plan.status()
    _check(bse, probs, refs, ds, 1e-6)
    plan.close()


# pair blocks of at least 64 x 64 rows: the second contraction runs on the
# tensor cores.  Nv = Nc = 8 puts the W^rr stage-1 side on (c, c') (tile rows
# from T), Nv = 8, Nc = 9 on (v, v') (tile rows from the other side, stored
# (c', c)); NG = 300 also cuts K into segments
@pytest.mark.parametrize("nv,nc,ng", [(8, 8, 59), (8, 8, 300), (8, 9, 59)], ids=str)
def test_tensor_core_stage2_matches_oracle_and_cuda_cores(bse, nv, nc, ng):
    import torch
    cfg = bi.BSEConfig(f"big-blocks-{nv}-{nc}-{ng}", grid=2, nv=nv, nc=nc, ng=ng, w_scale=0.05)
    p = bi.make_problem(cfg)
    A_ref, B_ref = O.build_A_B(p)
    ds, structs = _upload(bse, [p])
    tc = bse.Plan(structs, precision=bse.BSE_PREC_BF16X6)
    cc = bse.Plan(structs, precision=bse.BSE_PREC_BF16X6, tc_stage2=False)
    a = _build(bse, tc, ds)
    _check(bse, [p], [(A_ref, B_ref)], ds, 1e-6)
    b = _build(bse, cc, ds)
    _check(bse, [p], [(A_ref, B_ref)], ds, 1e-6)
    n = p["nk"] * p["nv"] * p["nc"]
    for x, y in zip(a, b):
        x = bse.matrix_to_numpy(x, n)
        y = bse.matrix_to_numpy(y, n)
        assert _rel(x, y) < 1e-6
    tc.close()
    cc.close()


@pytest.mark.parametrize("nv,nc,ng", [(8, 8, 300), (8, 9, 59)], ids=str)
def test_stage2_autotune(bse, nv, nc, ng):
    """The autotuner times the tensor-core stage 2 over its tile widths and
    pipeline depths: the chosen shape is one of the candidates, and the build
    matches the oracle and the default-shape build."""
    cfg = bi.BSEConfig(f"big-blocks-{nv}-{nc}-{ng}", grid=2, nv=nv, nc=nc, ng=ng, w_scale=0.05)
    p = bi.make_problem(cfg)
    A_ref, B_ref = O.build_A_B(p)
    ds, structs = _upload(bse, [p])
    plain = bse.Plan(structs, precision=bse.BSE_PREC_BF16X6)
    nt_d, st_d = plain.stage2_shape
    assert nt_d in (32, 64, 96, 128) and 2 <= st_d <= 6
    a = [x.clone() for x in _build(bse, plain, ds)]
    tuned = bse.Plan(structs, precision=bse.BSE_PREC_BF16X6, autotune=True)
    nt, st = tuned.stage2_shape
    assert nt in (32, nt_d) and st <= (st_d if nt == nt_d else 6) and st >= 2
    b = _build(bse, tuned, ds)
    _check(bse, [p], [(A_ref, B_ref)], ds, 1e-6)
    n = p["nk"] * p["nv"] * p["nc"]
    for x, y in zip(a, b):
        assert _rel(bse.matrix_to_numpy(x, n), bse.matrix_to_numpy(y, n)) < 1e-12
    # a plan without a tensor-core stage 2 reports none
    cc = bse.Plan(structs, precision=bse.BSE_PREC_BF16X6, tc_stage2=False)
    assert cc.stage2_shape == (0, 0)
    for pl in (plain, tuned, cc):
        pl.close()
