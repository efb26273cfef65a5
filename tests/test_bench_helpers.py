"""CPU checks of bench.py's host-side helpers: the FP32 CPU baseline, the
traffic record lookup (tied to the kernel source hash) and the reference
arm's JSON line."""
import importlib.util
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_cpu_fp32_baseline_reports_a_rate():
    b = load_bench()
    rng = np.random.default_rng(0)
    U = rng.standard_normal((300, 8)).astype(np.float32)
    I = rng.standard_normal((50, 8)).astype(np.float32)
    r = b.cpu_fp32_bmm(U, I, 5, target_s=0.05, block=64)
    assert r["value"] > 0 and r["unit"] == "users/s" and r["cores"] >= 1
    assert "not exact" in r["kind"]


def test_traffic_record_follows_the_kernel_source():
    b = load_bench()
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    key = "tc_score_select bf16 netflix-480189x17770 f=50 K=10"
    assert key in d and d[key]["bytes_per_launch"] > 0
    assert b.traffic_for(key, d[key]["source_hash"]) == d[key]["bytes_per_launch"]
    assert b.traffic_for(key, "0" * 16) is None
    assert b.traffic_for("no such kernel", d[key]["source_hash"]) is None


def test_walk_traffic_is_keyed_on_clusters_and_block():
    # a walk's DRAM traffic depends on |C| and the item block: the record of
    # one configuration is not reported for another
    b = load_bench()
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    stats = {"pairs_scored": 10 ** 9, "cand_emitted": 10 ** 6, "ms_kernel": 5.0}
    args = ("bf16", True, 51, 10 ** 6, 624961, 10, stats, PEAKS, "measured", 152, 2070.0, "kdd-1000000x624961")
    key = "tc_score_select walk bf16 kdd-1000000x624961 f=51 K=10 C=32 B=1024"
    assert key in d
    r = b.score_roofline(*args, (32, 1024))
    if d[key]["source_hash"] == b.kernel_source_hash(["tc_topk.cu", "tc_ptx.cuh", "tc_topk.h"]):
        assert r["traffic"] == d[key]["bytes_per_launch"]
    assert b.score_roofline(*args, (1024, 1024))["traffic"] is None
    assert b.score_roofline(*args, (32, 4096))["traffic"] is None


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "small-2048x1024-f32"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


PEAKS = {"hbm_gbs": 6781.8, "bf16_tflops": 1923.0, "sm_max_mhz": 2070.0}


def test_roofline_binds_on_the_slowest_ceiling():
    b = load_bench()
    # f = 10: 2 f FLOP per score is cheap, one issue slot per 32 scores binds
    sc = 480189 * 17770
    r = b.roofline("bf16", 10, sc, 1.0, 1e6, PEAKS, "measured", 152, 2070.0, "k x", ["tc_topk.cu"])
    t_sel = sc / (152 * 4 * 32 * 2070e6) * 1e3
    t_ten = 2 * 10 * sc / 1923e12 * 1e3
    assert r["ceiling"] == "select_issue" and r["bound"] == "alu"
    assert abs(r["ceilings_ms"]["select_issue"] - t_sel) < 1e-9 and abs(r["ceilings_ms"]["tensor"] - t_ten) < 1e-9
    assert abs(r["frac"] - t_sel / 1.0) < 1e-9
    # f = 100: the tensor ceiling binds; frac = achieved / peak
    r = b.roofline("bf16", 100, sc, 2.0, 1e6, PEAKS, "measured", 152, 2070.0, "k x", ["tc_topk.cu"])
    assert r["ceiling"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["frac"] - (2 * 100 * sc / 2e-3 / 1e12) / 1923.0) < 1e-9
    # a byte-heavy case binds on HBM
    r = b.roofline("bf16", 1, 1000, 1.0, 1e10, PEAKS, "measured", 152, 2070.0, "k x", ["tc_topk.cu"])
    assert r["ceiling"] == "hbm" and r["bound"] == "hbm"
    # FP32 CUDA-core form: the FMA peak from the SM count and clock
    r = b.roofline("fp32", 50, sc, 30.0, 1e6, PEAKS, "measured", 152, 2070.0, "k x", ["fp32_topk.cu"])
    assert r["ceiling"] == "alu_fp32_fma" and abs(r["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9


def test_exact_sample_reports_differences():
    b = load_bench()
    idx = np.arange(12, dtype=np.int32).reshape(4, 3)
    sc = np.linspace(1, 2, 12).reshape(4, 3)
    r = b.exact_sample(np.vstack([idx, idx]), np.vstack([sc, sc]), idx, sc)
    assert r == {"users": 4, "indices_equal": True, "rows_differing": 0, "max_rel_score_err": 0.0}
    j = idx.copy()
    j[2, 1] = 99
    s2 = sc.copy()
    s2[1, 0] *= 1 + 1e-7
    r = b.exact_sample(j, s2, idx, sc)
    assert not r["indices_equal"] and r["rows_differing"] == 1 and 0.9e-7 < r["max_rel_score_err"] < 1.1e-7
