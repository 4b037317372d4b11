#!/usr/bin/env python
"""Benchmark of the BSE hot path on one GB300 (or N, one process per GPU).

Default workload (the largest single-GPU configuration): the
molecular-crystal-like case, Q = 0, full BSE, Nk = 64 on a 4x4x4 grid,
Nv = Nc = 20, N = 25,600 (51,200 full), NG = 500, W with strong
off-diagonal structure; 39.8 GB of seeded synthetic inputs drawn on the GPU
and resident in HBM (far larger than the 129 MB L2).  One step = one build of
A and B (exchange + direct W^rr + direct W^ra + assembly) through a plan
created once (BF16x6 tensor-core contractions, FP64 assembly).

value: algorithmic build TFLOP/s (8 flops per complex multiply-add, no
padding, every (k, k') block counted) of the build, timed with CUDA events on
the launching stream.  ms_per_step: the build.  After the timed region, once:
the FP64 GPU build and the error of the mixed build against it; the time to
the lowest 16 excitons (mixed build + block Davidson with tensor-core
matvecs) against the plain FP64 GPU path (FP64 build + Davidson with FP64
matvecs); the end-to-end build through the public API from pinned host
buffers (inputs copied in, A and B copied out); the CPU oracle on sampled
(k, k') blocks; and, as extra keys, the optical-limit workload's (Nk = 64,
Nv = Nc = 4, N = 1,024, NG = 181) time to spectrum, mixed against FP64.
N > 1: every rank builds its own momentum transfer (Q replicas, no
collective), value sums the flops of all ranks over the slowest rank's time.

--config c1/c2/c3/c4/c4s select the other workloads.  --impl reference
times the CPU oracle (the plain FP64 restatement of the paper the CUDA path
is checked against) on the host cores, same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("BSE kernel-build TFLOP/s and time-to-spectrum, mixed vs FP64 GPU at "
          "≤1 meV error")
WORKLOAD = ("optical limit Q=0, full (non-TDA) BSE, Nk=64 (4x4x4), Nv=4, Nc=4, N=1024 "
            "(2048 full), NG=181")
WORKLOAD_C5 = ("molecular-crystal-like Q=0, full (non-TDA) BSE, Nk=64 (4x4x4), Nv=20, Nc=20, "
               "N=25600 (51200 full), NG=500, strong off-diagonal W")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
FP64_PEAK_TFLOPS = 1.25     # GB300 FP64 (CUDA-core and tensor) nominal rate
# eps by the Lanczos recursion: stop when eps changes by at most this fraction
# of max |eps| between checks (the 1e-3 bar at the peaks is far above it)
LANCZOS_TOL = 1e-6

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per build of a
# kernel phase, from one ncu capture of the kernel on the named workload,
# with a digest of the sources that kernel is compiled from: when those
# sources have changed since the capture the figure no longer describes the
# kernel and is reported as null.
KERNEL_SOURCES = ("paper_1904_05575_gb300/csrc/build_mixed.cu", "paper_1904_05575_gb300/csrc/tc_gemm.cuh",
                  "paper_1904_05575_gb300/csrc/tc_direct.cuh", "paper_1904_05575_gb300/csrc/bits.cuh",
                  "paper_1904_05575_gb300/csrc/bse_internal.h")
TRAFFIC = {
    # workload: {phase: (bytes per build, sources digest at capture)}
    "c5": {"mixed_stage2_tc": (49490195712, "dd6654958604b692"),
           "mixed_stage1_gemm": (26045644800, "dd6654958604b692"),
           "mixed_split": (50695242240, "dd6654958604b692"),
           "mixed_exchange": (13866989568, "dd6654958604b692"),
           "hermitian_complete": (20564305408, "dd6654958604b692")},
}


def sources_digest():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(workload):
    """{phase: bytes per build} of the captures still valid for the current sources."""
    dig = sources_digest()
    return {k: b for k, (b, sha) in TRAFFIC.get(workload, {}).items() if sha == dig}


def build_flops(nk, nv, nc, ng, coupling=True):
    """Algorithmic flops of one build: 8 per complex multiply-add, no padding.
    exchange 8 N^2 NG; W^rr stage 1 8 Nk^2 NG^2 min(nv^2, nc^2) + stage 2 8 NG N^2;
    W^ra stage 1 8 Nk^2 NG^2 nv nc + stage 2 8 NG N^2."""
    n = nk * nv * nc
    f = 8.0 * n * n * ng
    f += 8.0 * nk * nk * ng * ng * min(nv * nv, nc * nc) + 8.0 * ng * n * n
    if coupling:
        f += 8.0 * nk * nk * ng * ng * nv * nc + 8.0 * ng * n * n
    return f


def stage1_flops(nk, nv, nc, ng):
    return 8.0 * nk * nk * ng * ng * min(nv * nv, nc * nc), 8.0 * nk * nk * ng * ng * nv * nc


def built_pairs(nk, hermitian):
    """(k, k') blocks of a direct term the build computes: all Nk^2, or the
    Nk (Nk + 1) / 2 blocks k <= k' of a Hermitian plan."""
    return nk * (nk + 1) // 2 if hermitian else nk * nk


def split_bytes(nk, nv, nc, ng, pieces=3, hermitian=False, tc_stage2=None):
    """Bytes the operand split must move per build: every complex128 element
    read once (16 B) and written as BF16 planes over K padded to 16 (W rows
    padded to 32): 2 x pieces planes for a GEMM's row operand, 3 x pieces
    (-Im, Re, Im) for its column operand.  Rows: M_x twice (the exchange's
    row and column operands), W (once, or twice when W^rr applies it
    conjugate-transposed to the valence side; column operand), the stage-1
    side rows of both direct terms (row operand) and, for a term whose second
    contraction runs on the tensor cores, its other pair side (the column
    operand for W^rr with T on (c, c'), else the row operand)."""
    kp = -(-ng // 16) * 16
    ngp = -(-ng // 32) * 32
    n = nk * nv * nc
    npair = built_pairs(nk, hermitian)
    (rt_rr, rx_rr), (rt_ra, rx_ra) = term_rows(nv, nc)
    if tc_stage2 is None:
        tc_stage2 = min(rt_rr, rx_rr) >= 64
    w_splits = 1 if nc * nc <= nv * nv else 2
    a_rows = n + npair * (rt_rr + rt_ra)
    b_rows = n
    read_rows = 2 * n + npair * (rt_rr + rt_ra)
    if tc_stage2:
        read_rows += npair * (rx_rr + rx_ra)
        if nc * nc <= nv * nv:
            b_rows += npair * rx_rr
        else:
            a_rows += npair * rx_rr
        a_rows += npair * rx_ra
    read = 16 * ng * (read_rows + w_splits * nk * ng)
    write = 4 * pieces * kp * a_rows + 6 * pieces * kp * (b_rows + w_splits * nk * ngp)
    return read + write


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            out = {"source": "measured"}
            for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained"):
                if k in d:
                    out[k] = float(d[k])
            for k, v in FALLBACK_PEAKS.items():
                out.setdefault(k, v)
            return out
        except Exception:
            pass
    out = dict(FALLBACK_PEAKS)
    out["source"] = "fallback"
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(values, device, world):
    """Element-wise maximum of per-rank timings over all ranks (a no-op at
    world size 1); the only cross-rank exchange of the benchmark."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def weak_scaling_value(world, flops_per_rank, slowest_ms):
    """Whole-job TFLOP/s: every rank builds its own Q (replicas, no collective
    in the data path); the job takes as long as the slowest rank."""
    return world * flops_per_rank / (slowest_ms * 1e-3) / 1e12


def oracle_step(p, O):
    """One oracle pass over the workload: build, reduce, spectrum (seconds)."""
    t0 = time.perf_counter()
    A, B = O.build_A_B(p)
    t1 = time.perf_counter()
    O.spectrum(A, B, p)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def term_rows(nv, nc):
    """(rows_t, rows_x) of the W^rr and W^ra terms: stage 1 runs on the pair side
    with fewer rows (conduction pairs when nc^2 <= nv^2)."""
    rr = (nc * nc, nv * nv) if nc * nc <= nv * nv else (nv * nv, nc * nc)
    return rr, (nv * nc, nv * nc)


def upper_fraction(nk):
    """Share of the N^2 elements in the blocks k <= k' (the exchange of a
    whole problem with enough tiles, and every direct term of a Hermitian
    plan, computes those)."""
    return (nk + 1) / (2.0 * nk)


def build_rooflines(bse, prec, phases, steps, shapes, peaks, hermitian=False, workload=None,
                    upper_exchange=True):
    """Rooflines of the two longest build kernels (phases), from the
    library's CUDA-event phase timing over the timed region.  The work of
    each is what that kernel computes per build: the exchange over the blocks
    k <= k' (mirrors completed), the direct terms over all (k, k') blocks or,
    in a Hermitian plan, the blocks k <= k'."""
    def per_build(name):
        cnt, ms = phases.get(name, (0, float("nan")))
        return ms / steps
    if prec == bse.BSE_PREC_FP64:
        name = "fp64_wra_stage1"
        ra = sum(stage1_flops(*sh)[1] for sh in shapes)
        achieved = ra / (per_build(name) * 1e-3) / 1e12
        return ({"kernel": name, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                 "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                 "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak)",
                 "flops_per_launch": ra}, None)
    products = 6 if prec == bse.BSE_PREC_BF16X6 else 3
    pieces = 3 if prec == bse.BSE_PREC_BF16X6 else 2
    peak_t = peaks["bf16_tflops"] / products
    tensor_src = f"{peaks['source']} bf16 burst / {products} piece products"
    hbm_src = f"{peaks['source']} HBM copy bandwidth"
    s1 = s2 = ex = cmp_bytes = 0.0
    s2_term = [0.0, 0.0]
    for nk, nv, nc, ng in shapes:
        fr = built_pairs(nk, hermitian) / (nk * nk)
        n = nk * nv * nc
        s1 += fr * sum(stage1_flops(nk, nv, nc, ng))
        s2 += fr * 2 * 8.0 * ng * n * n
        ex += (upper_fraction(nk) if upper_exchange else 1.0) * 8.0 * n * n * ng
        # completion: the blocks k > k' of A and B read from their mirrors and written
        low = (1.0 - upper_fraction(nk)) * n * n
        cmp_bytes += 2 * 2 * 16 * low
        # CUDA-core stage 2 per term: X read as complex128, T as FP32 complex, the
        # A or B entries read and written once
        for i, (rt, rx) in enumerate(term_rows(nv, nc)):
            s2_term[i] += fr * (nk * nk * ng * (16 * rx + 8 * rt) + 32 * n * n)
    s2_bytes = sum(s2_term)
    kinds = {
        "mixed_direct_fused": ("gemm_split_bf16_direct: stage-1 GEMM + pair contraction, tcgen05",
                               "tensor", s1),
        "mixed_stage1_gemm": ("gemm_split_bf16: stage-1 GEMM, tcgen05", "tensor", s1),
        "mixed_stage2_tc": ("gemm_split_bf16: stage-2 pair-block GEMM, tcgen05", "tensor", s2),
        "mixed_exchange": ("gemm_split_bf16: exchange GEMM, tcgen05", "tensor", ex),
        "mixed_stage2": ("k_stage2 family: stage-2 contraction, CUDA cores", "hbm", s2_bytes),
        "mixed_stage2_wrr": ("k_stage2 family: W^rr stage-2 contraction, CUDA cores", "hbm",
                             s2_term[0]),
        "mixed_stage2_wra": ("k_stage2 family: W^ra stage-2 contraction, CUDA cores", "hbm",
                             s2_term[1]),
        "mixed_split": ("k_split: operand split, HBM pass", "hbm",
                        sum(split_bytes(*sh, pieces=pieces, hermitian=hermitian) for sh in shapes)),
        "hermitian_complete": ("k_hermitian_complete: blocks k > k' from their mirrors", "hbm",
                               cmp_bytes),
    }
    traffic = captured_traffic(workload) if workload else {}
    # the per-term stage-2 phases, where timed, replace their sum
    per_term = "mixed_stage2_wrr" in phases or "mixed_stage2_wra" in phases
    found = sorted(((per_build(k), k) for k in kinds
                    if k in phases and not (per_term and k == "mixed_stage2")), reverse=True)
    out = []
    for ms, name in found[:2]:
        what, bound, work = kinds[name]
        if bound == "tensor":
            achieved = work / (ms * 1e-3) / 1e12
            out.append({"kernel": f"{name} ({what})", "bound": "tensor", "achieved": achieved,
                        "peak": peak_t, "unit": "TFLOP/s", "frac": achieved / peak_t,
                        "traffic": traffic.get(name), "peak_source": tensor_src,
                        "flops_per_build": work, "ms_per_build": ms})
        else:
            achieved = work / (ms * 1e-3) / 1e9
            out.append({"kernel": f"{name} ({what})", "bound": "hbm", "achieved": achieved,
                        "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                        "traffic": traffic.get(name), "peak_source": hbm_src,
                        "bytes_per_build": work, "ms_per_build": ms})
    while len(out) < 2:
        out.append(None)
    return out[0], out[1]


def _host_block_view(p, rows, k, kp):
    """block_inputs for a problem drawn with k_rows=rows (pair arrays indexed
    by position in rows): the (k, k') block, k and k' both in rows."""
    import bse_inputs as bi
    r, rp = rows.index(k), rows.index(kp)
    h = dict(p, m_vv={(k, kp): p["m_vv"][r, kp]}, m_cc={(k, kp): p["m_cc"][r, kp]},
             n_vc={(k, kp): p["n_vc"][r, kp], (kp, k): p["n_vc"][rp, k]})
    return bi.block_inputs(h, k, kp)


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    import numpy as np
    import bse_inputs as bi
    from oracle import bse_oracle as O
    if args.config in ("c1", "c2"):
        p = bi.make_problem(args.config)
        flops = build_flops(p["nk"], p["nv"], p["nc"], p["ng"])
        for _ in range(args.warmup):
            oracle_step(p, O)
        tb, tt = [], []
        for _ in range(args.steps):
            b, t = oracle_step(p, O)
            tb.append(b)
            tt.append(t)
        value = flops / statistics.mean(tb) / 1e12
        ms = 1e3 * statistics.mean(tt)
        sample = f"full workload, {args.steps} steps of build+reduce+spectrum"
        workload = WORKLOAD if args.config == "c2" else args.config
    else:
        # the oracle on the (k, k') blocks among a few seeded k rows of the
        # workload (host generator, drawn once, untimed); a step is every
        # block among those rows, the build's flops scaled by blocks / Nk^2
        cfg = bi.CONFIGS[args.config]
        rng = np.random.default_rng(11)
        rows = sorted(int(x) for x in rng.choice(cfg.nk, size=min(4, cfg.nk), replace=False))
        p = bi.make_problem(cfg, k_rows=rows)
        blocks = [(k, kp) for k in rows for kp in rows]
        flops = build_flops(p["nk"], p["nv"], p["nc"], p["ng"]) * len(blocks) / p["nk"] ** 2
        views = [_host_block_view(p, rows, k, kp) for k, kp in blocks]
        for _ in range(args.warmup):
            for v in views:
                O.block_A_B(v)
        tb = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            for v in views:
                O.block_A_B(v)
            tb.append(time.perf_counter() - t0)
        value = flops / statistics.mean(tb) / 1e12
        ms = 1e3 * statistics.mean(tb)
        sample = (f"{len(blocks)} (k,k') blocks among k rows {rows} per step (block_A_B, numpy "
                  f"FP64), flops = the build's x {len(blocks)}/Nk^2")
        workload = WORKLOAD_C5 if args.config == "c5" else args.config
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "precision": "fp64 (numpy, host)"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cpu_cores(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_sampled_blocks(p, flops, shape_nk, seconds=10.0, label="Q 0"):
    """The oracle on seeded (k, k') blocks of a device-resident problem for
    about `seconds` of host time; algorithmic flops of a block = the build's
    over Nk^2."""
    import numpy as np
    import bse_inputs as bi
    from oracle import bse_oracle as O
    rng = np.random.default_rng(11)
    host = dict(p)
    for key in ("w", "m_x", "v_bar", "e_v", "e_c", "q_minus", "q_plus"):
        host[key] = p[key].cpu().numpy()
    nb, t_cpu = 0, 0.0
    while t_cpu < seconds and nb < 4096:
        k, kp = (int(x) for x in rng.integers(0, shape_nk, 2))
        blk = bi.block_inputs(host, k, kp)
        t0 = time.perf_counter()
        O.block_A_B(blk)
        t_cpu += time.perf_counter() - t0
        nb += 1
    return {"value": nb * flops / shape_nk ** 2 / t_cpu / 1e12, "unit": "TFLOP/s",
            "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{nb} seeded (k,k') blocks of {label} (block_A_B, numpy FP64)",
            "build_s": t_cpu}


def _rel_fro(X, Y, chunk=2048):
    """||X - Y||_F / ||Y||_F over the first n columns-major rows, in column
    chunks (no full-size temporaries)."""
    import torch
    num = den = 0.0
    for j in range(0, X.shape[0], chunk):
        a, b = X[j:j + chunk], Y[j:j + chunk]
        num += torch.linalg.norm(a - b).item() ** 2
        den += torch.linalg.norm(b).item() ** 2
    return (num / den) ** 0.5


def c2_time_to_spectrum(bse, bi, prec, steps=10, warmup=3):
    """The optical-limit workload's time to spectrum (mixed build + FP64
    reduction, eigensolve, spectrum) against the plain FP64 GPU path, and
    the energy error between them."""
    import torch
    stream = torch.cuda.current_stream()
    p = bi.make_problem("c2")
    nk, nv, nc, ng = p["nk"], p["nv"], p["nc"], p["ng"]
    n = nk * nv * nc
    d = bse.upload_problem(p)
    st = bse.make_problem_struct(d)
    S = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    L = torch.empty_like(S)
    E = torch.empty(n, dtype=torch.float64, device="cuda")
    osc = torch.empty_like(E)
    om = torch.as_tensor(p["omega"]).cuda()
    eps = torch.empty(len(p["omega"]), dtype=torch.complex128, device="cuda")
    rho = torch.as_tensor(p["rho"]).cuda()
    vc = nk * p["omega_cell"]
    plan = bse.Plan([st], precision=prec, autotune=True)

    def run(fp64):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        if fp64:
            bse.bse_build_kernel([st], bse.BSE_PREC_FP64)
        else:
            plan.execute()
        e1.record(stream)
        bse.bse_reduce(n, d["A"], d["B"], S, L)
        bse.bse_spectrum(n, S, L, rho, p["c_q"], vc, om, p["delta"], E, osc, eps)
        e2.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), e0.elapsed_time(e2)

    eps_lz = torch.empty_like(eps)

    def run_lanczos():
        # eps only: mixed build + the Lanczos recursion (no reduction, no eigensolve)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.execute()
        # FP64 products: at N = 1,024 the tensor-core products' per-call set-up
        # costs more than they save (160 against 46 ms per eps)
        k = bse.bse_spectrum_lanczos(n, d["A"], d["B"], rho, p["c_q"], vc, om, p["delta"], eps_lz,
                                     tol=LANCZOS_TOL, matvec_precision=bse.BSE_PREC_FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), k

    for _ in range(warmup):
        run(False)
    mixed = [run(False) for _ in range(steps)]
    E_mixed = E.clone()
    run_lanczos()
    lanczos = [run_lanczos() for _ in range(steps)]
    run(True)
    fp64 = [run(True) for _ in range(3)]
    plan.status()
    plan.close()
    t_mx = statistics.mean(x[1] for x in mixed)
    t_64 = statistics.mean(x[1] for x in fp64)
    t_lz = statistics.mean(x[0] for x in lanczos)
    y = eps.imag.cpu().numpy()
    pk = [i for i in range(1, len(y) - 1) if y[i] > y[i - 1] and y[i] >= y[i + 1] and y[i] > 0.1 * y.max()]
    e_lz = eps_lz.cpu().numpy()
    lz = {"method": ("mixed build + Lanczos recursion on (A-B)(A+B), eps only (no eigensolve), "
                     "FP64 products"),
          "time_to_eps_ms": t_lz, "lanczos_steps": lanczos[-1][1],
          "speedup_vs_fp64_time_to_spectrum": t_64 / t_lz,
          "max_rel_dIm_eps_at_peaks_vs_fp64": float(max(
              (abs(e_lz.imag[i] - y[i]) / abs(y[i]) for i in pk), default=0.0))}
    return {"workload": WORKLOAD, "build_ms": statistics.mean(x[0] for x in mixed),
            "build_tflops": build_flops(nk, nv, nc, ng) / (statistics.mean(x[0] for x in mixed)
                                                           * 1e-3) / 1e12,
            "time_to_spectrum_ms": t_mx, "fp64_build_ms": statistics.mean(x[0] for x in fp64),
            "fp64_time_to_spectrum_ms": t_64, "speedup_time_to_spectrum": t_64 / t_mx,
            "max_dE_meV_vs_fp64": (E_mixed - E).abs().max().item() * 1e3,
            "eps_by_lanczos": lz}


def run_headline(args, bse, bi, prec, world, rank, local):
    """The largest single-GPU workload (c5), build-only steps; see the module
    docstring."""
    import torch
    dev = "cuda"
    stream = torch.cuda.current_stream()
    seed = 20190411 + rank
    herm = not args.all_blocks
    p = bi.make_problem_torch(args.config, q_index=args.q, seed=seed)
    nk, nv, nc, ng = p["nk"], p["nv"], p["nc"], p["ng"]
    n = nk * nv * nc
    flops = build_flops(nk, nv, nc, ng)
    d = bse.upload_problem(p)
    st = bse.make_problem_struct(d)
    torch.cuda.synchronize()
    plan = bse.Plan([st], precision=prec, autotune=True, hermitian=herm)
    for _ in range(args.warmup):
        plan.execute()
    torch.cuda.synchronize()
    plan.status()

    # ---- timed region: `steps` builds ----
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = bse.bse_kernel_launches()
    bse.bse_phase_timing(True)
    for e0, e1 in evs:
        e0.record(stream)
        plan.execute()
        e1.record(stream)
    torch.cuda.synchronize()
    bse.bse_phase_timing(False)
    launches = bse.bse_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    plan.status()
    phases = bse.bse_phase_report()
    build_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    t_build = max_over_ranks([statistics.mean(build_ms)], dev, world)[0]
    value = weak_scaling_value(world, flops, t_build)
    computed = flops
    if herm:   # direct terms over the blocks k <= k' (both stages)
        fr = built_pairs(nk, True) / nk ** 2
        s1 = sum(stage1_flops(nk, nv, nc, ng))
        s2 = 2 * 8.0 * ng * n * n
        computed = flops - (1 - fr) * (s1 + s2)
    computed -= (1 - upper_fraction(nk)) * 8.0 * n * n * ng   # exchange over k <= k'
    extra = {"build_ms": t_build, "build_ms_min": min(build_ms),
             "computed_flops_per_build": computed,
             "computed_tflops": computed / (t_build * 1e-3) / 1e12,
             "build_api": ("bse_plan_execute (plan created once, "
                           + ("BSE_PLAN_HERMITIAN: direct terms over the blocks k <= k', "
                              "the rest completed from the mirrors; " if herm else "")
                           + f"autotuned: stage-1 tiles of {plan.tile_cols} columns, "
                           + "stage-2 tiles of {} columns, {}-deep pipeline)".format(*plan.stage2_shape)),
             "phase_ms_per_step": {k: v[1] / args.steps for k, v in phases.items()}}

    # ---- once: the plain FP64 GPU build and the error against it ----
    E_mx = torch.empty(args.nev, dtype=torch.float64, device=dev)
    E_64 = torch.empty(args.nev, dtype=torch.float64, device=dev)
    A64, B64 = torch.empty_like(d["A"]), torch.empty_like(d["B"])
    st64 = bse.make_problem_struct(dict(d, A=A64, B=B64))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bse.bse_build_kernel([st64], bse.BSE_PREC_FP64)
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = e0.elapsed_time(e1)
    extra.update({"fp64_build_ms": fp64_ms,
                  "fp64_build_tflops": flops / (fp64_ms * 1e-3) / 1e12,
                  "speedup_vs_fp64_build": fp64_ms / t_build,
                  "A_rel_fro_vs_fp64": _rel_fro(d["A"], A64),
                  "B_rel_fro_vs_fp64": _rel_fro(d["B"], B64)})

    # ---- once: time to the lowest excitons, mixed against plain FP64 ----
    if args.nev > 0:
        tol = args.dav_tol or 1e-5
        runs, iters = [], 0
        for _ in range(2):      # the first call also sets up the matvec workspace
            e0.record(stream)
            plan.execute()
            iters = bse.bse_lowest_excitons(n, d["A"], d["B"], args.nev, E_mx, None, tol_ev=tol,
                                            max_iter=args.dav_max_iter, matvec_precision=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            runs.append(e0.elapsed_time(e1))
        e0.record(stream)
        iters64 = bse.bse_lowest_excitons(n, A64, B64, args.nev, E_64, None, tol_ev=tol,
                                          max_iter=args.dav_max_iter,
                                          matvec_precision=bse.BSE_PREC_FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        dav64 = e0.elapsed_time(e1)
        extra["lowest_excitons"] = {
            "nev": args.nev, "residual_tol_ev": tol,
            "method": "mixed build + block Davidson (tensor-core matvecs, diagonal preconditioner)",
            "time_to_lowest_excitons_ms": runs[-1], "first_call_ms": runs[0],
            "davidson_iterations": iters,
            "fp64_method": "FP64 build + block Davidson (FP64 matvecs)",
            "fp64_time_to_lowest_excitons_ms": fp64_ms + dav64, "fp64_davidson_iterations": iters64,
            "speedup_vs_fp64": (fp64_ms + dav64) / runs[-1],
            "max_dE_meV_vs_fp64": (E_mx - E_64).abs().max().item() * 1e3,
            "lowest_E_eV": [round(x, 6) for x in E_mx[:4].tolist()]}
    del A64, B64, st64
    torch.cuda.empty_cache()

    # ---- once: time to eps_M on the grid by the Lanczos recursion (mixed
    # build, then no reduction and no eigensolve) ----
    if not args.no_lanczos:
        om = torch.as_tensor(p["omega"]).to(dev)
        rho = p["rho"] if torch.is_tensor(p["rho"]) else torch.as_tensor(p["rho"]).to(dev)
        eps_lz = torch.empty(len(p["omega"]), dtype=torch.complex128, device=dev)
        lz_ms, lz_steps = [], 0
        for _ in range(2):
            e0.record(stream)
            plan.execute()
            lz_steps = bse.bse_spectrum_lanczos(n, d["A"], d["B"], rho, p["c_q"],
                                                nk * p["omega_cell"], om, p["delta"], eps_lz,
                                                tol=LANCZOS_TOL, matvec_precision=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            lz_ms.append(e0.elapsed_time(e1))
        extra["eps_by_lanczos"] = {
            "method": ("mixed build + Lanczos recursion on (A-B)(A+B), eps only (no eigensolve), "
                       "products split once and run on the tensor cores"),
            "time_to_eps_ms": lz_ms[-1], "lanczos_steps": lz_steps, "tol": LANCZOS_TOL}

    # ---- end to end through the public API with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        keys = ("e_v", "e_c", "m_x", "m_vv", "m_cc", "n_vc", "w", "q_minus", "q_plus", "v_bar")
        host = {}
        for k in keys:
            host[k] = torch.empty(d[k].shape, dtype=d[k].dtype, pin_memory=True)
            host[k].copy_(d[k])
        A_h = torch.empty(d["A"].shape, dtype=d["A"].dtype, pin_memory=True)
        B_h = torch.empty(d["B"].shape, dtype=d["B"].dtype, pin_memory=True)
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = 2 * A_h.numel() * A_h.element_size()
        e2e_ms = []
        for i in range(1 + args.e2e_steps):
            e0.record(stream)
            for k, t in host.items():
                d[k].copy_(t, non_blocking=True)
            plan.execute()
            A_h.copy_(d["A"], non_blocking=True)
            B_h.copy_(d["B"], non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            if i > 0:
                e2e_ms.append(e0.elapsed_time(e1))
        plan.status()
        t_e2e = max_over_ranks([statistics.mean(e2e_ms)], dev, world)[0]
        e2e = {"value": weak_scaling_value(world, flops, t_e2e), "unit": "TFLOP/s",
               "ms_per_step": t_e2e, "steps": args.e2e_steps,
               "what": "inputs copied in from pinned host memory, build, A and B copied out",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        del host, A_h, B_h

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sampled_blocks(p, flops, nk, label=f"Q {args.q}")

    peaks = load_peaks()
    roofline, roofline_secondary = build_rooflines(bse, prec, phases, args.steps,
                                                   [(nk, nv, nc, ng)], peaks, hermitian=herm,
                                                   workload=args.config)
    plan.close()
    del d, p, st
    torch.cuda.empty_cache()
    if not args.no_c2:
        extra["optical_limit_c2"] = c2_time_to_spectrum(bse, bi, prec)

    if rank == 0:
        input_gb = 16 * (n * ng + 3 * nk * nk * nv * nc * ng + nk * ng * ng) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_build,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "bf16x6": "bf16x6(f32 acc)", "bf16x3": "bf16x3(f32 acc)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD_C5 if args.config == "c5" else args.config,
                       "precision": args.precision, "step": "one build of A and B",
                       "hermitian_plan": herm,
                       "l2": f"inputs larger than L2 ({input_gb:.1f} GB resident in HBM)",
                       "parallelism": f"Q replicas x{world}"},
            "roofline": roofline, "roofline_secondary": roofline_secondary,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches, "peaks": peaks,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    return 0


def _eps_peaks(eps_im, omega):
    """Local maxima of Im eps above 10 % of its largest value."""
    import numpy as np
    y = np.asarray(eps_im)
    idx = [i for i in range(1, len(y) - 1) if y[i] > y[i - 1] and y[i] >= y[i + 1]
           and y[i] > 0.1 * y.max()]
    return idx


def _dense_lowest(bse, n, A, B, nev):
    """Lowest nev pairs (E, X+Y [nev, n]) of A, B by the FP64 dense route:
    reduction, full eigensolve, X+Y of the lowest."""
    import torch
    S = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    L = torch.empty_like(S)
    bse.bse_reduce(n, A, B, S, L)
    E = torch.empty(n, dtype=torch.float64, device="cuda")
    osc = torch.empty_like(E)
    rho = torch.zeros(n, dtype=torch.complex128, device="cuda")
    bse.bse_spectrum(n, S, L, rho, 1.0, 1.0, None, 0.05, E, osc, None)
    X = torch.empty((nev, n), dtype=torch.complex128, device="cuda")
    bse.bse_xpy(n, nev, S, L, E[:nev].contiguous(), X)
    return E[:nev].contiguous(), X


def run_mlp_family(args, bse, bi, prec, world, rank, local):
    """The learned Davidson preconditioner on a family of problems along Q
    (every Q drawn from the streams of Q index 0, so only v(G+Q) and c_Q change):
    the middle Q of the configuration's line is the unseen one, the other four
    train the 10-feature network.  Per training Q: the dense FP64 solve's
    lowest nev pairs, then a Davidson trajectory started from the nearest
    training Q's X+Y with features from the two nearest.  At the unseen Q: the
    Davidson iterations and times of the diagonal preconditioner from a cold
    start and from the nearest Q's X+Y, and of the trained network from the
    same start, each against the dense solve's energies."""
    import torch
    if args.config not in ("c4s", "c2", "c1"):
        raise SystemExit("--mlp-family draws whole problems: use c4s (or c1 / c2)")
    cfg = bi.CONFIGS[args.config]
    nq = len(cfg.q_abs)
    test_q = nq // 2
    pool = [q for q in range(nq) if q != test_q]
    near = lambda q, k: sorted([j for j in pool if j != q],
                               key=lambda j: abs(cfg.q_abs[j] - cfg.q_abs[q]))[:k]
    nev, tol = args.nev, args.dav_tol or 1e-4
    stream = torch.cuda.current_stream()
    built, pairs = {}, {}
    for q in range(nq):
        p = bi.make_problem_torch(args.config, q_index=q, draws_of=0, seed=20190411 + rank)
        d = bse.upload_problem(p)
        n = p["nk"] * p["nv"] * p["nc"]
        plan = bse.Plan([bse.make_problem_struct(d)], precision=prec, hermitian=True)
        plan.execute()
        plan.status()
        plan.close()
        built[q] = (d["A"], d["B"])
        pairs[q] = _dense_lowest(bse, n, d["A"], d["B"], nev)
        del d, p
    torch.cuda.empty_cache()
    net = bse.MLP(seed=5, n_features=10)
    F, C, W = [], [], []
    t0 = time.perf_counter()
    for q in pool:
        net.set_neighbours(torch.stack([pairs[j][1] for j in near(q, 2)]))
        f, c, w = bse.bse_mlp_trajectory_samples(n, *built[q], *pairs[q], tol_ev=tol, max_iter=80,
                                                 capacity=min(1 << 22, 160 * nev * n), mlp=net,
                                                 start=pairs[near(q, 1)[0]][1])
        F.append(f)
        C.append(c)
        W.append(w)
    F, C, W = (torch.cat(x).contiguous() for x in (F, C, W))
    t_samples = time.perf_counter() - t0
    L0, _ = net.loss_grad(F, C, W)
    t0 = time.perf_counter()
    L1 = net.train(F, C, W, 600, 2e-3)
    t_train = time.perf_counter() - t0
    nbs = near(test_q, 2)
    net.set_neighbours(torch.stack([pairs[j][1] for j in nbs]))
    start = pairs[nbs[0]][1]
    E_ref = pairs[test_q][0]
    runs = {}
    for name, pc, st in (("diagonal_cold", 0, None), ("diagonal_from_nearest_q", 0, start),
                         ("learned_from_nearest_q", 1, start)):
        E = torch.empty(nev, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        converged = True
        try:
            it = bse.bse_lowest_excitons(n, *built[test_q], nev, E, None, tol_ev=tol,
                                         max_iter=args.dav_max_iter, precond=pc,
                                         mlp=net if pc else None, matvec_precision=prec, start=st)
        except bse.BSEError as err:     # E holds the last Ritz values
            if err.status != bse.BSE_ERR_NO_CONV:
                raise
            converged, it = False, args.dav_max_iter
        e1.record(stream)
        torch.cuda.synchronize()
        runs[name] = {"iterations": it, "converged": converged, "ms": e0.elapsed_time(e1),
                      "max_dE_meV_vs_dense": (E - E_ref).abs().max().item() * 1e3}
    if rank == 0:
        print(json.dumps({"metric": "learned Davidson preconditioner at an unseen Q",
                          "config": args.config, "n": n, "nev": nev, "residual_tol_ev": tol,
                          "q_abs": list(cfg.q_abs), "unseen_q_index": test_q,
                          "training_q_indices": pool, "samples": int(C.numel()),
                          "sampling_s": t_samples, "training_s": t_train,
                          "training_loss": [L0, L1], "runs": runs}), flush=True)
    return 0


def run_eps_lanczos(args, bse, bi, prec, world, rank, local):
    """eps_M at one Q by the mixed build + the Lanczos recursion against the
    plain FP64 GPU path (FP64 build, reduction, eigensolve, spectrum): the
    largest relative difference of Im eps at its peaks and of eps on the grid,
    and both times to eps."""
    import numpy as np
    import torch
    q = args.eps_lanczos
    stream = torch.cuda.current_stream()
    p = bi.make_problem_torch(args.config, q_index=q, seed=20190411 + rank)
    n = p["nk"] * p["nv"] * p["nc"]
    d = bse.upload_problem(p)
    st = bse.make_problem_struct(d)
    om = torch.as_tensor(p["omega"]).cuda()
    rho = p["rho"] if torch.is_tensor(p["rho"]) else torch.as_tensor(p["rho"]).cuda()
    vc = p["nk"] * p["omega_cell"]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    eps64 = torch.empty(len(p["omega"]), dtype=torch.complex128, device="cuda")
    ev[0].record(stream)
    bse.bse_build_kernel([st], bse.BSE_PREC_FP64)
    S = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    L = torch.empty_like(S)
    E = torch.empty(n, dtype=torch.float64, device="cuda")
    osc = torch.empty_like(E)
    bse.bse_reduce(n, d["A"], d["B"], S, L)
    bse.bse_spectrum(n, S, L, rho, p["c_q"], vc, om, p["delta"], E, osc, eps64)
    ev[1].record(stream)
    torch.cuda.synchronize()
    del S, L
    torch.cuda.empty_cache()
    plan = bse.Plan([st], precision=prec, hermitian=True)
    eps = torch.empty_like(eps64)
    ev[2].record(stream)
    plan.execute()
    steps = bse.bse_spectrum_lanczos(n, d["A"], d["B"], rho, p["c_q"], vc, om, p["delta"], eps,
                                     tol=1e-8, matvec_precision=prec)
    ev[3].record(stream)
    torch.cuda.synchronize()
    plan.status()
    plan.close()
    r, e = eps64.cpu().numpy(), eps.cpu().numpy()
    pk = _eps_peaks(r.imag, p["omega"])
    row = {"metric": "eps_M by Lanczos (mixed build) vs the FP64 GPU path", "config": args.config,
           "q_index": q, "n": n, "lanczos_steps": steps, "peaks": len(pk),
           "max_rel_dIm_eps_at_peaks": float(max((abs(e.imag[i] - r.imag[i]) / abs(r.imag[i])
                                                  for i in pk), default=0.0)),
           "max_rel_d_eps": float(np.abs(e - r).max() / np.abs(r).max()),
           "fp64_time_to_eps_ms": ev[0].elapsed_time(ev[1]),
           "lanczos_time_to_eps_ms": ev[2].elapsed_time(ev[3])}
    if rank == 0:
        print(json.dumps(row), flush=True)
    return 0


def run_eps_qs(args, bse, bi, prec, world, rank, local):
    """eps_M at several momentum transfers of a workload, the mixed path (split-
    precision Hermitian plan + FP64 reduction, eigensolve and spectrum) against
    the plain FP64 GPU path (FP64 build + the same FP64 steps): per Q the
    largest exciton-energy difference, the largest relative difference of
    Im eps_M at its peaks (local maxima above 10 % of the largest) and of the
    peak positions, and the times.  Each Q's inputs are drawn on the GPU;
    each path's dense reduction and eigensolve is done once."""
    import numpy as np
    import torch
    qs = [int(x) for x in args.eps_qs.split(",")]
    stream = torch.cuda.current_stream()
    rows = []
    for q in qs:
        p = bi.make_problem_torch(args.config, q_index=q, seed=20190411 + rank)
        nk, nv, nc, ng = p["nk"], p["nv"], p["nc"], p["ng"]
        n = nk * nv * nc
        d = bse.upload_problem(p)
        st = bse.make_problem_struct(d)
        om = torch.as_tensor(p["omega"]).cuda()
        rho = p["rho"] if torch.is_tensor(p["rho"]) else torch.as_tensor(p["rho"]).cuda()
        vc = nk * p["omega_cell"]
        S = torch.empty((n, n), dtype=torch.complex128, device="cuda")
        L = torch.empty_like(S)
        out = {}
        for name in ("fp64", "mixed"):
            E = torch.empty(n, dtype=torch.float64, device="cuda")
            osc = torch.empty_like(E)
            eps = torch.empty(len(p["omega"]), dtype=torch.complex128, device="cuda")
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            if name == "fp64":
                bse.bse_build_kernel([st], bse.BSE_PREC_FP64)
            else:
                plan = bse.Plan([st], precision=prec, hermitian=True)
                ev[0].record(stream)
                plan.execute()
                plan.status()
            ev[1].record(stream)
            bse.bse_reduce(n, d["A"], d["B"], S, L)
            bse.bse_spectrum(n, S, L, rho, p["c_q"], vc, om, p["delta"], E, osc, eps)
            ev[2].record(stream)
            torch.cuda.synchronize()
            if name == "mixed":
                plan.close()
            out[name] = {"E": E.cpu().numpy(), "eps": eps.cpu().numpy(),
                         "build_ms": ev[0].elapsed_time(ev[1]), "total_ms": ev[0].elapsed_time(ev[2])}
        ef, em = out["fp64"]["E"], out["mixed"]["E"]
        pf = _eps_peaks(out["fp64"]["eps"].imag, p["omega"])
        imf, imm = out["fp64"]["eps"].imag, out["mixed"]["eps"].imag
        pm = _eps_peaks(imm, p["omega"])
        dpos = max((abs(p["omega"][a] - p["omega"][b]) for a, b in zip(pf, pm)), default=0.0) \
            if len(pf) == len(pm) else float("nan")
        rows.append({"q_index": q, "q_abs": float(np.linalg.norm(p["q_vec"])), "n": n,
                     "max_dE_meV": float(np.abs(ef - em).max() * 1e3),
                     "lowest_E_eV": float(ef[0]),
                     "peaks": len(pf),
                     "max_rel_dIm_eps_at_peaks": float(max((abs(imm[i] - imf[i]) / abs(imf[i])
                                                            for i in pf), default=0.0)),
                     "max_rel_d_eps": float(np.abs(out["mixed"]["eps"] - out["fp64"]["eps"]).max()
                                            / np.abs(out["fp64"]["eps"]).max()),
                     "peak_shift_eV": dpos,
                     "fp64_build_ms": out["fp64"]["build_ms"], "mixed_build_ms": out["mixed"]["build_ms"],
                     "fp64_total_ms": out["fp64"]["total_ms"], "mixed_total_ms": out["mixed"]["total_ms"]})
        print(json.dumps(rows[-1]), flush=True)
        del S, L, d, p, st
        torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps({"metric": "eps_M, mixed vs FP64 GPU path", "config": args.config,
                          "rows": rows}), flush=True)
    return 0


def run_c3_all(args, bse, bi, prec, world, rank, local):
    """All 16 momentum transfers of the finite-momentum batch (Nk = 512 on an
    8x8x8 grid, NG = 113, uneven (Nv, Nc) windows, N from 2,048 to 12,288):
    their 326 GB of complex128 inputs exceed the device, so the Q are packed
    in order into groups of at most --c3-group-gb of inputs; each group's
    inputs are drawn on the GPU (untimed) and built by one Hermitian plan
    (every Q's exchange tiles in one persistent launch, all its direct terms
    in the next), executed `warmup` times and timed `steps` times.  A step
    is the build of all 16 Q: ms_per_step is the sum over groups of the mean
    group time."""
    import torch
    cfg = bi.CONFIGS["c3"]
    nq = len(cfg.q_abs)
    seed = 20190411 + rank
    stream = torch.cuda.current_stream()
    unit = cfg.nk * cfg.nk * cfg.ng * 16

    def qbytes(q):
        nv, nc = cfg.window(q)
        return unit * (nv * nv + nc * nc + nv * nc)

    groups, cur, cur_b = [], [], 0.0
    for q in range(nq):
        if cur and cur_b + qbytes(q) > args.c3_group_gb * 1e9:
            groups.append(cur)
            cur, cur_b = [], 0.0
        cur.append(q)
        cur_b += qbytes(q)
    groups.append(cur)
    sampler = ClockSampler(local)
    sampler.start()
    total_ms, flops, launches, per_group = 0.0, 0.0, 0, []
    phases_all = {}
    for g in groups:
        probs = [bi.make_problem_torch(cfg, q_index=q, seed=seed) for q in g]
        ds = [bse.upload_problem(p) for p in probs]
        sts = [bse.make_problem_struct(d) for d in ds]
        torch.cuda.synchronize()
        plan = bse.Plan(sts, precision=prec, autotune=True, hermitian=not args.all_blocks)
        for _ in range(args.warmup):
            plan.execute()
        torch.cuda.synchronize()
        plan.status()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        l0 = bse.bse_kernel_launches()
        bse.bse_phase_timing(True)
        for e0, e1 in evs:
            e0.record(stream)
            plan.execute()
            e1.record(stream)
        torch.cuda.synchronize()
        bse.bse_phase_timing(False)
        launches += bse.bse_kernel_launches() - l0
        plan.status()
        for k, v in bse.bse_phase_report().items():
            c, ms = phases_all.get(k, (0, 0.0))
            phases_all[k] = (c + v[0], ms + v[1])
        ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs)
        f = sum(build_flops(p["nk"], p["nv"], p["nc"], p["ng"]) for p in probs)
        per_group.append({"q": g, "windows": [list(cfg.window(q)) for q in g],
                          "n": [p["nk"] * p["nv"] * p["nc"] for p in probs],
                          "input_gb": round(sum(qbytes(q) for q in g) / 1e9, 1),
                          "build_ms": ms, "tflops": f / (ms * 1e-3) / 1e12})
        total_ms += ms
        flops += f
        plan.close()
        del plan, sts, ds, probs
        torch.cuda.empty_cache()
    clocks = sampler.stop()
    t = max_over_ranks([total_ms], "cuda", world)[0]
    value = weak_scaling_value(world, flops, t)
    peaks = load_peaks()
    shapes = [(cfg.nk,) + tuple(cfg.window(q)) + (cfg.ng,) for q in range(nq)]
    roofline, roofline_secondary = build_rooflines(bse, prec, phases_all, args.steps, shapes, peaks,
                                                   hermitian=not args.all_blocks, workload="c3")
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "bf16x6": "bf16x6(f32 acc)", "bf16x3": "bf16x3(f32 acc)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "finite-momentum batch: all 16 Q along [100], Nk=512 (8x8x8), "
                                   "NG=113, uneven windows, N 2048..12288, built in groups of Q "
                                   "(inputs drawn on the GPU per group)",
                       "precision": args.precision, "hermitian_plan": not args.all_blocks,
                       "l2": "inputs larger than L2 (tens of GB per group)",
                       "parallelism": f"Q replicas x{world}"},
            "groups": per_group,
            "phase_ms_per_step": {k: v[1] / args.steps for k, v in phases_all.items()},
            "roofline": roofline, "roofline_secondary": roofline_secondary,
            "cpu_baseline": None, "e2e": None, "clocks": clocks, "gpu_launches": launches,
            "peaks": peaks,
        }
        print(json.dumps(line), flush=True)
    return 0


def run_c4(args, bse, bi, prec, world, rank, local):
    """Core-level workload (c4: Nk=512, Nv=2 core levels, Nc=20, NG=300,
    N=20,480, full BSE; c4s: the same recipe on a 4x4x4 grid): c4's pair
    arrays (m_cc alone 503 GB) exceed the device memory, so A and B are built
    in k-row slabs of --slab-rows rows.  Before each slab's
    build its m_vv and m_cc are drawn on the device (untimed, S3 kept across
    slabs); n_vc, W, M_x and A, B stay resident.  Each slab's plan execute is
    timed `steps` times after `warmup` untimed runs; a step is the whole build,
    so ms_per_step is the sum over slabs of the mean slab time.  --lowest then
    runs block Davidson (tensor-core matvecs) on the complete A, B; with
    --fp64-dense the plain FP64 path (FP64 slab builds + dense reduction and
    eigensolve) is timed beside it and the exciton energies compared."""
    import numpy as np
    import torch
    dev = "cuda"
    stream = torch.cuda.current_stream()
    seed = 20190411 + rank
    kn = args.slab_rows
    p = bi.make_problem_torch(args.config, q_index=0, seed=seed, k_slab=(0, kn))
    nk, nv, nc, ng = p["nk"], p["nv"], p["nc"], p["ng"]
    n = nk * nv * nc
    flops = build_flops(nk, nv, nc, ng)
    d = bse.upload_problem(p)
    fp64_dense = args.lowest and args.fp64_dense
    if fp64_dense:
        A64, B64 = torch.zeros_like(d["A"]), torch.zeros_like(d["B"])
    slab_ms, fp64_slab_ms, tile_cols = [], [], None
    launches = 0
    sampler = ClockSampler(local)
    sampler.start()
    if nk % kn:
        raise SystemExit(f"--slab-rows {kn} must divide Nk = {nk}")
    for kb in range(0, nk, kn):
        if kb:
            for x in (p, d):
                x["m_vv"] = x["m_cc"] = None
            torch.cuda.empty_cache()
            p["m_vv"], p["m_cc"] = d["m_vv"], d["m_cc"] = bi.pair_slab_torch(args.config, kb, kn, 0,
                                                                               seed)
        plan = bse.Plan([bse.make_problem_struct(d, k_begin=kb, k_count=kn)], precision=prec,
                        autotune=True)
        tile_cols = plan.tile_cols
        for _ in range(args.warmup):
            plan.execute()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        l0 = bse.bse_kernel_launches()
        bse.bse_phase_timing(True)
        for e0, e1 in evs:
            e0.record(stream)
            plan.execute()
            e1.record(stream)
        torch.cuda.synchronize()
        bse.bse_phase_timing(False)
        launches += bse.bse_kernel_launches() - l0
        plan.status()
        plan.close()
        slab_ms.append(statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs))
        if fp64_dense:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            st64 = bse.make_problem_struct(dict(d, A=A64, B=B64), k_begin=kb, k_count=kn)
            e0.record(stream)
            bse.bse_build_kernel([st64], bse.BSE_PREC_FP64)
            e1.record(stream)
            torch.cuda.synchronize()
            fp64_slab_ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    phases = bse.bse_phase_report()
    m_cc_gb = kn * nk * nc * nc * ng * 16 / 1e9
    t_build = max_over_ranks([sum(slab_ms)], dev, world)[0]
    value = weak_scaling_value(world, flops, t_build)

    # CPU oracle on seeded (k, k') blocks of the last slab's rows, about 10 s
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import bse_oracle as O
        host = dict(p)
        for key in ("w", "m_x", "v_bar", "e_v", "e_c", "q_minus", "q_plus"):
            host[key] = p[key].cpu().numpy()
        kb_last = nk - kn
        rng = np.random.default_rng(11)
        nb, t_cpu = 0, 0.0
        while t_cpu < 10.0 and nb < 4096:
            k, kp = kb_last + int(rng.integers(0, kn)), int(rng.integers(0, nk))
            blk_host = dict(host, m_vv={(k, kp): p["m_vv"][k - kb_last, kp]},
                            m_cc={(k, kp): p["m_cc"][k - kb_last, kp]})
            blk = bi.block_inputs(blk_host, k, kp)
            t0 = time.perf_counter()
            O.block_A_B(blk)
            t_cpu += time.perf_counter() - t0
            nb += 1
        cpu = {"value": nb * flops / nk ** 2 / t_cpu / 1e12, "unit": "TFLOP/s",
               "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{nb} seeded (k,k') blocks of the last slab (block_A_B, numpy FP64)",
               "build_s": t_cpu}

    extra = {}
    if args.lowest:
        for x in (p, d):
            for key in ("m_vv", "m_cc", "n_vc", "w"):
                x[key] = None
        torch.cuda.empty_cache()
        nev = min(args.nev, n)
        E_dav = torch.empty(nev, dtype=torch.float64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tol = args.dav_tol or 1e-4
        converged = True
        e0.record(stream)
        try:
            iters = bse.bse_lowest_excitons(n, d["A"], d["B"], nev, E_dav, None, tol_ev=tol,
                                            max_iter=args.dav_max_iter, matvec_precision=prec)
        except bse.BSEError as err:     # E_dav still holds the last Ritz values
            if err.status != bse.BSE_ERR_NO_CONV:
                raise
            converged, iters = False, args.dav_max_iter
        e1.record(stream)
        torch.cuda.synchronize()
        dav = e0.elapsed_time(e1)
        low = {"nev": nev, "method": "mixed slab builds + block Davidson (tensor-core matvecs, "
                                     "diagonal preconditioner)",
               "time_to_lowest_excitons_ms": t_build + dav, "davidson_ms": dav,
               "davidson_iterations": iters, "residual_tol_ev": tol, "converged": converged,
               "lowest_E_eV": [round(x, 6) for x in E_dav[:4].tolist()]}
        if fp64_dense:
            del d["A"], d["B"]
            torch.cuda.empty_cache()
            S2 = torch.empty((n, n), dtype=torch.complex128, device=dev)
            L2 = torch.empty_like(S2)
            E_all = torch.empty(n, dtype=torch.float64, device=dev)
            osc_all = torch.empty_like(E_all)
            om = torch.as_tensor(p["omega"]).to(dev)
            eps = torch.empty(len(p["omega"]), dtype=torch.complex128, device=dev)
            e0.record(stream)
            bse.bse_reduce(n, A64, B64, S2, L2)
            bse.bse_spectrum(n, S2, L2, p["rho"], p["c_q"], nk * p["omega_cell"], om, p["delta"],
                             E_all, osc_all, eps)
            e1.record(stream)
            torch.cuda.synchronize()
            fp64_total = sum(fp64_slab_ms) + e0.elapsed_time(e1)
            low.update({"fp64_build_ms": sum(fp64_slab_ms), "fp64_dense_ms": fp64_total,
                        "speedup_vs_fp64_dense": fp64_total / low["time_to_lowest_excitons_ms"],
                        "max_dE_meV_vs_fp64_dense": (E_dav - E_all[:nev]).abs().max().item() * 1e3})
        extra["lowest_excitons"] = low

    peaks = load_peaks()
    roofline, roofline_secondary = build_rooflines(bse, prec, phases, args.steps,
                                                   [(nk, nv, nc, ng)], peaks, workload=args.config,
                                                   upper_exchange=False)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_build,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "bf16x6": "bf16x6(f32 acc)", "bf16x3": "bf16x3(f32 acc)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"{args.config} core-level case: Q 0, Nk={nk}, Nv={nv} core levels, "
                                   f"Nc={nc}, N={n}, NG={ng}, full BSE, built in {nk // kn} k-row "
                                   f"slabs of {kn} (pair arrays drawn on the GPU per slab)",
                       "precision": args.precision, "build_only": True,
                       "l2": f"inputs larger than L2 ({m_cc_gb:.1f} GB of m_cc per slab)",
                       "parallelism": f"Q replicas x{world}"},
            "build_ms": t_build, "slab_build_ms": slab_ms,
            "build_api": f"bse_plan_execute per slab (tile width autotuned: {tile_cols} columns)",
            "phase_ms_per_step": {k: v[1] / args.steps for k, v in phases.items()},
            "roofline": roofline, "roofline_secondary": roofline_secondary,
            "cpu_baseline": cpu, "e2e": None, "clocks": clocks,
            "gpu_launches": launches, "peaks": peaks,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c5",
                    help="c5 (default: the largest single-GPU workload), c1, c2, c3, c4, c4s")
    ap.add_argument("--q", type=int, default=0, help="c5: the momentum transfer index built")
    ap.add_argument("--all-blocks", action="store_true",
                    help="c5: compute every (k, k') block (no BSE_PLAN_HERMITIAN)")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="c5: timed end-to-end steps (after one untimed)")
    ap.add_argument("--eps-lanczos", type=int, default=None,
                    help="one Q index: eps by mixed build + Lanczos against the FP64 GPU path")
    ap.add_argument("--no-lanczos", action="store_true",
                    help="c5: skip timing eps by the Lanczos recursion")
    ap.add_argument("--mlp-family", action="store_true",
                    help="learned Davidson preconditioner trained at four Q of a family, "
                         "judged at the fifth (c4s)")
    ap.add_argument("--eps-qs", default=None,
                    help="comma-separated Q indices: eps_M of the mixed path against the plain "
                         "FP64 GPU path at each (dense reduction and eigensolve per path)")
    ap.add_argument("--c3-group-gb", type=float, default=120.0,
                    help="c3 --qs all: complex128 input gigabytes per group of Q")
    ap.add_argument("--no-c2", action="store_true",
                    help="c5: skip the optical-limit time-to-spectrum extra keys")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "bf16x6", "bf16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--build-only", action="store_true",
                    help="time the build alone (no reduction / eigensolve / spectrum)")
    ap.add_argument("--qs", default="0", help="comma-separated Q indices built by one plan")
    ap.add_argument("--device-inputs", action="store_true",
                    help="draw the inputs on the GPU (automatic for c3 and c5)")
    ap.add_argument("--nev", type=int, default=None,
                    help="lowest excitons for time-to-lowest-excitons (16; 50 for c4)")
    ap.add_argument("--lowest", action="store_true",
                    help="build-only configs: also time mixed build + Davidson (tensor-core matvecs)")
    ap.add_argument("--dav-tol", type=float, default=None,
                    help="Davidson residual tolerance in eV (1e-5; 1e-4 for c4, whose "
                         "interaction terms reach 100 eV)")
    ap.add_argument("--dav-max-iter", type=int, default=300)
    ap.add_argument("--slab-rows", type=int, default=64,
                    help="c4 / c4s: k rows per slab of the pair arrays")
    ap.add_argument("--fp64-dense", action="store_true",
                    help="with --lowest: also time the plain FP64 path (FP64 build + dense solve)")
    args = ap.parse_args()
    if args.nev is None:
        args.nev = 50 if args.config in ("c4", "c4s") else 16
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)

    import numpy as np
    import torch

    import bse_inputs as bi
    import paper_1904_05575_gb300 as bse
    from paper_1904_05575_gb300 import build as _build

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    bse.load()

    prec_map = {"fp64": bse.BSE_PREC_FP64, "bf16x6": bse.BSE_PREC_BF16X6,
                "bf16x3": bse.BSE_PREC_BF16X3}
    if args.precision == "auto":
        args.precision = "bf16x6" if bse.mixed_available() else "fp64"
    prec = prec_map[args.precision]

    # each rank: its own momentum transfers (Q replicas), resident in HBM
    if args.mlp_family:
        rc = run_mlp_family(args, bse, bi, prec, world, rank, local)
        return rc
    if args.eps_lanczos is not None:
        return run_eps_lanczos(args, bse, bi, prec, world, rank, local)
    if args.eps_qs:
        rc = run_eps_qs(args, bse, bi, prec, world, rank, local)
        if world > 1:
            dist.destroy_process_group()
        return rc
    if args.config in ("c5", "c5s"):
        rc = run_headline(args, bse, bi, prec, world, rank, local)
        if world > 1:
            dist.destroy_process_group()
        return rc
    if args.config == "c3" and args.qs == "all":
        rc = run_c3_all(args, bse, bi, prec, world, rank, local)
        if world > 1:
            dist.destroy_process_group()
        return rc
    if args.config in ("c4", "c4s"):
        rc = run_c4(args, bse, bi, prec, world, rank, local)
        if world > 1:
            dist.destroy_process_group()
        return rc
    qs = [int(x) for x in args.qs.split(",")]
    device_inputs = args.device_inputs or args.config in ("c3", "c5")
    if device_inputs or len(qs) > 1:
        args.build_only = True       # spectra of N up to 25,600 take minutes in cuSOLVER
    if device_inputs:
        probs = [bi.make_problem_torch(args.config, q_index=q, seed=20190411 + rank) for q in qs]
    else:
        probs = [bi.make_problem(args.config, q_index=q, seed=20190411 + rank) for q in qs]
    p = probs[0]
    nk, nv, nc, ng = p["nk"], p["nv"], p["nc"], p["ng"]
    n = nk * nv * nc
    shapes = [(pp["nk"], pp["nv"], pp["nc"], pp["ng"]) for pp in probs]
    flops = sum(build_flops(*sh) for sh in shapes)
    ds = [bse.upload_problem(pp) for pp in probs]
    sts = [bse.make_problem_struct(dd) for dd in ds]
    d, st = ds[0], sts[0]
    dev = "cuda"
    nsq = 0 if args.build_only else n
    S = torch.empty((nsq, nsq), dtype=torch.complex128, device=dev)
    L = torch.empty_like(S)
    E = torch.empty(n, dtype=torch.float64, device=dev)
    osc = torch.empty_like(E)
    om = torch.as_tensor(p["omega"]).to(dev)
    eps = torch.empty(len(p["omega"]), dtype=torch.complex128, device=dev)
    rho = p["rho"] if torch.is_tensor(p["rho"]) else torch.as_tensor(p["rho"]).to(dev)
    vc = nk * p["omega_cell"]
    stream = torch.cuda.current_stream()

    # a plan per precision (validation, grouping, scratch and tensor maps once,
    # outside the timed region); each step's build is the plan's execute
    plans = {prec: bse.Plan(sts, precision=prec, autotune=True)}

    def step(precision, ev=None):
        if ev:
            ev[0].record(stream)
        if precision not in plans:
            plans[precision] = bse.Plan(sts, precision=precision)
        plans[precision].execute()
        if ev:
            ev[1].record(stream)
        if not args.build_only:
            bse.bse_reduce(n, d["A"], d["B"], S, L)
            bse.bse_spectrum(n, S, L, rho, p["c_q"], vc, om, p["delta"], E, osc, eps)
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step(prec)
    torch.cuda.synchronize()
    plans[prec].status()

    # ---- timed region ----
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = bse.bse_kernel_launches()
    bse.bse_phase_timing(True)
    for i in range(args.steps):
        step(prec, evs[i])
    torch.cuda.synchronize()
    bse.bse_phase_timing(False)
    launches = bse.bse_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    plans[prec].status()          # bounded device waits all completed
    phases = bse.bse_phase_report()
    build_ms = [e[0].elapsed_time(e[1]) for e in evs]
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    t_build, t_step = max_over_ranks([statistics.mean(build_ms), statistics.mean(step_ms)],
                                     dev, world)
    value = weak_scaling_value(world, flops, t_build)

    # accuracy of this precision against the FP64 GPU build (same inputs)
    E_this = E.clone()
    A_this = d["A"].clone()
    extra = {}
    if prec != bse.BSE_PREC_FP64 and not args.build_only:
        fp_ms = []
        for i in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bse.bse_build_kernel([st], bse.BSE_PREC_FP64)   # plain FP64 GPU build, one call
            e1.record(stream)
            torch.cuda.synchronize()
            fp_ms.append(e0.elapsed_time(e1))
        bse.bse_reduce(n, d["A"], d["B"], S, L)
        bse.bse_spectrum(n, S, L, rho, p["c_q"], vc, om, p["delta"], E, osc, eps)
        torch.cuda.synchronize()
        dA = (torch.linalg.norm(A_this - d["A"]) / torch.linalg.norm(d["A"])).item()
        dE = (E_this - E).abs().max().item() * 1e3
        extra = {"fp64_build_ms": statistics.mean(fp_ms),
                 "fp64_build_tflops": flops / (statistics.mean(fp_ms) * 1e-3) / 1e12,
                 "speedup_vs_fp64_build": statistics.mean(fp_ms) / t_build,
                 "A_rel_fro_vs_fp64": dA, "max_dE_meV_vs_fp64": dE}
        fp64_t2s = []       # plain FP64 GPU path: build + reduction + eigensolve + spectrum
        for i in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bse.bse_build_kernel([st], bse.BSE_PREC_FP64)
            bse.bse_reduce(n, d["A"], d["B"], S, L)
            bse.bse_spectrum(n, S, L, rho, p["c_q"], vc, om, p["delta"], E, osc, eps)
            e1.record(stream)
            torch.cuda.synchronize()
            fp64_t2s.append(e0.elapsed_time(e1))
        E_fp64 = E.clone()
        extra["fp64_time_to_spectrum_ms"] = statistics.mean(fp64_t2s)
        extra["speedup_time_to_spectrum"] = statistics.mean(fp64_t2s) / t_step

        # ---- time to the lowest excitons: mixed build + block Davidson against
        # the plain FP64 GPU path (build + dense reduction + eigensolve) ----
        if args.nev > 0:
            nev = min(args.nev, n)
            E_dav = torch.empty(nev, dtype=torch.float64, device=dev)
            dav_ms, iters = [], 0
            for i in range(4):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plans[prec].execute()
                iters = bse.bse_lowest_excitons(n, d["A"], d["B"], nev, E_dav, None,
                                                tol_ev=1e-5, max_iter=300)
                e1.record(stream)
                torch.cuda.synchronize()
                if i > 0:
                    dav_ms.append(e0.elapsed_time(e1))
            t_dav = statistics.mean(dav_ms)
            # the other route: mixed build + dense reduction / eigensolve (the
            # timed step, which yields every exciton)
            best = min(t_dav, t_step)
            extra["lowest_excitons"] = {
                "nev": nev, "time_to_lowest_excitons_ms": best,
                "method": "mixed build + block Davidson" if t_dav <= t_step else
                          "mixed build + dense reduction and eigensolve",
                "davidson_ms": t_dav, "davidson_iterations": iters,
                "davidson_preconditioner": "diagonal", "dense_mixed_ms": t_step,
                "fp64_dense_ms": statistics.mean(fp64_t2s),
                "speedup_vs_fp64_dense": statistics.mean(fp64_t2s) / best,
                "max_dE_meV_davidson_vs_fp64_dense":
                    (E_dav - E_fp64[:nev]).abs().max().item() * 1e3,
                "max_dE_meV_dense_mixed_vs_fp64_dense": dE}

    # ---- large N: time to the lowest excitons by mixed build + Davidson with
    # tensor-core matvecs, against the plain FP64 path (FP64 build + dense
    # reduction and eigensolve) when asked ----
    if args.build_only and args.lowest and len(probs) == 1:
        nev = min(args.nev, n)
        E_dav = torch.empty(nev, dtype=torch.float64, device=dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plans[prec].execute()
        iters = bse.bse_lowest_excitons(n, d["A"], d["B"], nev, E_dav, None, tol_ev=1e-5,
                                        max_iter=300, matvec_precision=prec)
        e1.record(stream)
        torch.cuda.synchronize()
        low = {"nev": nev, "method": "mixed build + block Davidson (tensor-core matvecs)",
               "time_to_lowest_excitons_ms": e0.elapsed_time(e1), "davidson_iterations": iters}
        if args.fp64_dense:
            S2 = torch.empty((n, n), dtype=torch.complex128, device=dev)
            L2 = torch.empty_like(S2)
            E_all = torch.empty(n, dtype=torch.float64, device=dev)
            osc_all = torch.empty_like(E_all)
            e0.record(stream)
            bse.bse_build_kernel([st], bse.BSE_PREC_FP64)
            e1.record(stream)
            bse.bse_reduce(n, d["A"], d["B"], S2, L2)
            bse.bse_spectrum(n, S2, L2, rho, p["c_q"], vc, om, p["delta"], E_all, osc_all, eps)
            e2 = torch.cuda.Event(enable_timing=True)
            e2.record(stream)
            torch.cuda.synchronize()
            low.update({"fp64_build_ms": e0.elapsed_time(e1), "fp64_dense_ms": e0.elapsed_time(e2),
                        "speedup_vs_fp64_dense": e0.elapsed_time(e2) / low["time_to_lowest_excitons_ms"],
                        "max_dE_meV_vs_fp64_dense": (E_dav - E_all[:nev]).abs().max().item() * 1e3})
            del S2, L2
        extra["lowest_excitons"] = low

    # ---- roofline of the dominant build kernel (phase timing, live) ----
    peaks = load_peaks()
    roofline, roofline_secondary = build_rooflines(bse, prec, phases, args.steps, shapes, peaks,
                                                   workload=args.config,
                                                   upper_exchange=sum(sh[0] * sh[1] * sh[2]
                                                                      for sh in shapes) >= 2048)

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not args.no_e2e and not args.build_only:
        host = {k: d[k].cpu().pin_memory() for k in
                ("e_v", "e_c", "m_x", "m_vv", "m_cc", "n_vc", "w", "q_minus", "q_plus", "v_bar")}
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        E_h = torch.empty(n, dtype=torch.float64).pin_memory()
        osc_h = torch.empty_like(E_h).pin_memory()
        eps_h = torch.empty(len(p["omega"]), dtype=torch.complex128).pin_memory()
        d2h = (E_h.numel() + osc_h.numel()) * 8 + eps_h.numel() * 16
        e2e_ms = []
        for i in range(args.warmup + args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k, t in host.items():
                d[k].copy_(t, non_blocking=True)
            step(prec)
            E_h.copy_(E, non_blocking=True)
            osc_h.copy_(osc, non_blocking=True)
            eps_h.copy_(eps, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= args.warmup:
                e2e_ms.append(e0.elapsed_time(e1))
        t_e2e = max_over_ranks([statistics.mean(e2e_ms)], dev, world)[0]
        e2e = {"value": weak_scaling_value(world, flops, t_e2e), "unit": "TFLOP/s",
               "ms_per_step": t_e2e, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- CPU oracle on the host cores (rank 0, N = 1 only), bounded sample ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import bse_oracle as O
        if device_inputs:
            # oracle on seeded (k, k') blocks for about 10 s; algorithmic flops
            # of a block = the build's over Nk^2
            rng = np.random.default_rng(11)
            host = dict(p)
            for key in ("w", "m_x", "v_bar", "e_v", "e_c", "q_minus", "q_plus"):
                host[key] = p[key].cpu().numpy()
            nb, t_cpu = 0, 0.0
            while t_cpu < 10.0 and nb < 4096:
                k, kp = (int(x) for x in rng.integers(0, nk, 2))
                blk = bi.block_inputs(host, k, kp)
                t0 = time.perf_counter()
                O.block_A_B(blk)
                t_cpu += time.perf_counter() - t0
                nb += 1
            cpu = {"value": nb * build_flops(*shapes[0]) / nk ** 2 / t_cpu / 1e12,
                   "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"{nb} seeded (k,k') blocks of Q {qs[0]} (block_A_B, numpy FP64)",
                   "build_s": t_cpu}
        else:
            tb, _ = oracle_step(p, O)
            cpu = {"value": flops / tb / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(),
                   "kind": "oracle", "sample": "one full build of the same workload (numpy FP64)",
                   "build_s": tb}

    if rank == 0:
        input_gb = sum(t.numel() * t.element_size() for dd in ds for key, t in dd.items()
                       if key in ("m_x", "m_vv", "m_cc", "n_vc", "w")) / 1e9
        phase_ms = {k: v[1] / args.steps for k, v in phases.items()}
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "bf16x6": "bf16x6(f32 acc)", "bf16x3": "bf16x3(f32 acc)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD if args.config == "c2" else
                       f"{args.config}: Q {qs}, windows {[(pp['nv'], pp['nc']) for pp in probs]}, "
                       f"Nk={nk}, NG={ng}" + (" (inputs drawn on the GPU)" if device_inputs else ""),
                       "precision": args.precision, "build_only": args.build_only,
                       "l2": f"inputs larger than L2 ({input_gb:.2f} GB resident per step)",
                       "parallelism": f"Q replicas x{world}"},
            "build_ms": t_build, "time_to_spectrum_ms": t_step,
            "build_api": "bse_plan_execute (plan created once, tile width autotuned: "
                         f"{plans[prec].tile_cols} columns)",
            "phase_ms_per_step": phase_ms,
            "roofline": roofline, "roofline_secondary": roofline_secondary,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches, "peaks": peaks,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
