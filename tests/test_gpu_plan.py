"""Batched plans: several momentum transfers with uneven band windows built by
one plan, against the oracle; the plan's execute captured in a CUDA graph and
replayed; the tile-width autotuner (GPU)."""
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
