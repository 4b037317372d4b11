"""Builds at the full sizes of the larger workloads, checked on sampled blocks.

The inputs are drawn on the GPU (bse_inputs.make_problem_torch: the recipe of
the CPU generator, tens of GB), built through an autotuned plan as the
benchmark does, and every sampled (k, k') block of A and B is compared with
the oracle's block_A_B evaluated on that block's inputs copied back to the
host.  Errors are relative Frobenius norms over the union of the sampled
blocks; the diagonal blocks carry E^ip, so the off-diagonal blocks (pure
interaction terms) are also checked on their own.

  c5  Nk = 64, Nv = Nc = 20, N = 25,600, NG = 500 (strong off-diagonal W), Q = 0
  c3  Nk = 512, NG = 113, two of the 16 Q in one plan: the smallest window
      (2, 2), N = 2,048, and the largest (4, 6), N = 12,288, at |Q| = 0.1 and 1.5
  c4  Nk = 512, Nv = 2 core levels, Nc = 20, NG = 300, N = 20,480: m_cc alone
      is 503 GB, so A and B are built in k-row slabs of 64 rows (two slabs
      built: the first and a middle one) and sampled blocks of their rows
      are checked
"""
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


def _sample_blocks(nk, s, n_diag=3, seed=5, entries=50_000):
    """3 diagonal blocks and enough seeded off-diagonal blocks of s x s
    entries for about `entries` sampled entries (9 to 2000 blocks)."""
    n_off = int(min(2000, max(9, entries // (s * s)), nk * (nk - 1)))
    rng = np.random.default_rng(seed)
    diag = sorted({0, nk // 2, nk - 1})[:n_diag]
    out = [(k, k) for k in diag]
    while len(out) < n_diag + n_off:
        k, kp = (int(x) for x in rng.integers(0, nk, 2))
        if k != kp and (k, kp) not in out:
            out.append((k, kp))
    return out


def _block(t, k, kp, s):
    """(k, k') block of a column-major [n, ld] tensor as numpy rows (v, c)."""
    return t[kp * s:(kp + 1) * s, k * s:(k + 1) * s].cpu().numpy().T


def _host_view(p):
    """The problem with its small arrays copied to the host once (W, M_x, ...);
    the pair arrays stay on the device and are read block by block."""
    out = dict(p)
    for k in ("w", "m_x", "v_bar", "e_v", "e_c", "q_minus", "q_plus"):
        out[k] = p[k].cpu().numpy()
    return out


def _errors(p, d, blocks):
    p = _host_view(p)
    s = p["nv"] * p["nc"]
    num = {"A": 0.0, "B": 0.0, "A_off": 0.0}
    den = {"A": 0.0, "B": 0.0, "A_off": 0.0}
    for k, kp in blocks:
        a_ref, b_ref = O.block_A_B(bi.block_inputs(p, k, kp))
        a, b = _block(d["A"], k, kp, s), _block(d["B"], k, kp, s)
        for key, x, r in (("A", a, a_ref), ("B", b, b_ref)) + ((("A_off", a, a_ref),) if k != kp else ()):
            num[key] += np.linalg.norm(x - r) ** 2
            den[key] += np.linalg.norm(r) ** 2
    return {key: float(np.sqrt(num[key] / den[key])) for key in num}


def _free(*objs):
    import torch
    for o in objs:
        if isinstance(o, dict):
            o.clear()
    torch.cuda.empty_cache()


def test_c5_full_size_bf16x6_plan(bse):
    import torch
    p = bi.make_problem_torch("c5", q_index=0)
    d = bse.upload_problem(p)
    plan = bse.Plan([bse.make_problem_struct(d)], precision=bse.BSE_PREC_BF16X6, autotune=True)
    plan.execute()
    plan.status()
    torch.cuda.synchronize()
    blocks = _sample_blocks(p["nk"], p["nv"] * p["nc"])
    err = _errors(p, d, blocks)
    print(f"\nc5 {len(blocks)} sampled blocks: rel Frobenius {err}, tile cols {plan.tile_cols}, "
          f"fused {plan.fused}")
    plan.close()
    _free(d, p)
    assert err["A"] < 1e-6 and err["B"] < 1e-6 and err["A_off"] < 1e-6, err


@pytest.mark.parametrize("prec,tol", [(2, 1e-6), (0, 1e-12)], ids=["bf16x6", "fp64"])
def test_c3_full_size_uneven_windows_one_plan(bse, prec, tol):
    import torch
    qs = (0, 15)
    probs = [bi.make_problem_torch("c3", q_index=q) for q in qs]
    assert [(p["nv"], p["nc"]) for p in probs] == [(2, 2), (4, 6)]
    ds = [bse.upload_problem(p) for p in probs]
    plan = bse.Plan([bse.make_problem_struct(d) for d in ds], precision=prec, autotune=(prec != 0))
    plan.execute()
    plan.status()
    torch.cuda.synchronize()
    for q, p, d in zip(qs, probs, ds):
        blocks = _sample_blocks(p["nk"], p["nv"] * p["nc"], seed=q)
        err = _errors(p, d, blocks)
        print(f"\nc3 Q{q} window ({p['nv']},{p['nc']}) N={p['nk'] * p['nv'] * p['nc']}, "
              f"{len(blocks)} blocks: {err}")
        assert err["A"] < tol and err["B"] < tol and err["A_off"] < tol, err
    plan.close()
    for d in ds:
        _free(d)
    for p in probs:
        _free(p)


class _SlabRows:
    """A slab's m_vv or m_cc indexed with whole-problem k (for block_inputs)."""

    def __init__(self, t, k_begin):
        self.t, self.k_begin = t, k_begin

    def __getitem__(self, idx):
        k, kp = idx
        return self.t[k - self.k_begin, kp]


def _sample_slab_blocks(nk, s, kb, kn, seed, entries=50_000):
    """3 diagonal blocks of the slab's rows and seeded off-diagonal blocks (k, k')
    with k in the slab, about `entries` sampled entries."""
    rng = np.random.default_rng(seed)
    out = [(k, k) for k in sorted({kb, kb + kn // 2, kb + kn - 1})]
    n_off = int(min(2000, max(9, entries // (s * s))))
    while len(out) < 3 + n_off:
        k, kp = kb + int(rng.integers(0, kn)), int(rng.integers(0, nk))
        if k != kp and (k, kp) not in out:
            out.append((k, kp))
    return out


def test_c4_full_size_bf16x6_slabs(bse):
    import time
    import torch
    kn = 64
    p = bi.make_problem_torch("c4", q_index=0, k_slab=(0, kn))
    nk, s = p["nk"], p["nv"] * p["nc"]
    d = bse.upload_problem(p)
    for kb in (0, 320):
        if kb:
            for x in (p, d):
                x["m_vv"] = x["m_cc"] = None
            torch.cuda.empty_cache()
            m_vv, m_cc = bi.pair_slab_torch("c4", kb, kn, q_index=0)
            p["m_vv"], p["m_cc"] = d["m_vv"], d["m_cc"] = m_vv, m_cc
        plan = bse.Plan([bse.make_problem_struct(d, k_begin=kb, k_count=kn)],
                        precision=bse.BSE_PREC_BF16X6, autotune=True)
        plan.execute()
        plan.status()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.execute()
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0)
        plan.status()
        plan.close()
        view = dict(p)
        view["m_vv"], view["m_cc"] = _SlabRows(p["m_vv"], kb), _SlabRows(p["m_cc"], kb)
        blocks = _sample_slab_blocks(nk, s, kb, kn, seed=kb)
        err = _errors(view, d, blocks)
        print(f"\nc4 slab [{kb}, {kb + kn}) build {ms:.1f} ms, {len(blocks)} sampled blocks: {err}")
        assert err["A"] < 1e-6 and err["B"] < 1e-6 and err["A_off"] < 1e-6, err
    _free(d, p)
