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


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "small-2048x1024-f32"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
