"""bench.py on the CPU: the oracle arm's JSON line (--impl reference) and the
roofline bookkeeping of the GPU arm, fed with made-up phase timings."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--config", "c1", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "TFLOP/s" and line["higher_is_better"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["steps"] == 1 and line["warmup"] == 3


class _FakeLib:
    BSE_PREC_FP64, BSE_PREC_BF16X6, BSE_PREC_BF16X3 = 0, 2, 3


def test_rooflines_per_term_and_traffic(monkeypatch):
    import bench
    peaks = {"source": "measured", "hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
             "bf16_tflops_sustained": 1700.0}
    shapes = [(512, 2, 20, 300)]
    # per build (steps = 2): W^rr stage 2 100 ms, W^ra 50 ms, their sum 150 ms, stage 1 50 ms
    phases = {"mixed_stage2_wrr": (16, 200.0), "mixed_stage2_wra": (16, 100.0),
              "mixed_stage2": (2, 300.0), "mixed_stage1_gemm": (16, 100.0)}
    # a capture taken from the current sources is reported; one from other sources is not
    monkeypatch.setitem(bench.TRAFFIC, "c4", {"mixed_stage2_wrr": (5.3e11, bench.sources_digest()),
                                              "mixed_stage2_wra": (8.7e10, "0" * 16)})
    r1, r2 = bench.build_rooflines(_FakeLib, 2, phases, 2, shapes, peaks, workload="c4",
                                   upper_exchange=False)
    # the per-term phases replace their sum; the longest comes first
    assert r1["kernel"].startswith("mixed_stage2_wrr") and r1["bound"] == "hbm"
    assert r2["kernel"].startswith("mixed_stage2_wra") or r2["kernel"].startswith("mixed_stage1")
    nk, nv, nc, ng = shapes[0]
    n = nk * nv * nc
    wrr_bytes = nk * nk * ng * (16 * nc * nc + 8 * nv * nv) + 32 * n * n
    assert abs(r1["bytes_per_build"] - wrr_bytes) < 1.0
    assert abs(r1["achieved"] - wrr_bytes / 0.1 / 1e9) < 1e-6 * r1["achieved"]
    assert r1["traffic"] == 5.3e11
    if r2["kernel"].startswith("mixed_stage2_wra"):
        assert r2["traffic"] is None           # stale digest
    # other workloads carry no captured traffic
    r3, _ = bench.build_rooflines(_FakeLib, 2, phases, 2, [(8, 2, 20, 59)], peaks)
    assert r3["traffic"] is None


def test_rooflines_fused_c2():
    import bench
    peaks = {"source": "measured", "hbm_gbs": 6800.0, "bf16_tflops": 1932.0,
             "bf16_tflops_sustained": 1700.0}
    phases = {"mixed_direct_fused": (4, 1.6), "mixed_split": (24, 0.8), "mixed_exchange": (4, 0.2)}
    r1, r2 = bench.build_rooflines(_FakeLib, 2, phases, 4, [(64, 4, 4, 181)], peaks)
    assert r1["kernel"].startswith("mixed_direct_fused") and r1["bound"] == "tensor"
    flops = sum(bench.stage1_flops(64, 4, 4, 181))
    assert abs(r1["achieved"] - flops / 0.4e-3 / 1e12) < 1e-9 * r1["achieved"]
    assert abs(r1["peak"] - 1932.0 / 6) < 1e-9
    assert r2["kernel"].startswith("mixed_split") and r2["bound"] == "hbm"


def test_rooflines_hermitian_work():
    """A Hermitian plan computes the direct terms over Nk (Nk + 1) / 2 of the
    Nk^2 blocks: the stage-2 roofline counts that work, the exchange the
    blocks k <= k', and the split the pair rows actually split."""
    import bench
    peaks = {"source": "measured", "hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
             "bf16_tflops_sustained": 1700.0}
    nk, nv, nc, ng = 64, 20, 20, 500
    n = nk * nv * nc
    phases = {"mixed_stage2_tc": (1, 30.0), "mixed_stage1_gemm": (1, 20.0),
              "mixed_exchange": (1, 8.0), "mixed_split": (9, 7.0), "hermitian_complete": (2, 3.0)}
    r1, r2 = bench.build_rooflines(_FakeLib, 2, phases, 1, [(nk, nv, nc, ng)], peaks,
                                   hermitian=True)
    assert r1["kernel"].startswith("mixed_stage2_tc")
    assert abs(r1["flops_per_build"] - (nk + 1) / (2 * nk) * 2 * 8.0 * ng * n * n) < 1.0
    assert r2["kernel"].startswith("mixed_stage1_gemm")
    full = sum(bench.stage1_flops(nk, nv, nc, ng))
    assert abs(r2["flops_per_build"] - full * 2080 / 4096) < 1.0
    assert bench.split_bytes(nk, nv, nc, ng, hermitian=True) < 0.6 * bench.split_bytes(nk, nv, nc, ng)


def test_reference_arm_sampled_blocks():
    """The oracle arm on a workload too large for a whole host build: blocks
    among a few seeded k rows per step."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--config", "c4s", "--steps", "2", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    assert "blocks among k rows" in line["cpu_baseline"]["sample"]
    assert line["e2e"]["value"] == line["value"]
