"""Benchmark: exact batch top-K MIPS throughput (users/sec) on GB300.

Default workload: the KDD shape -- 1,000,000 clustered users x 624,961
items, f = 51, K = 10 -- searched with Maximus (Sec. III, Algorithm 1) with
its cluster count |C| and item block B picked by the library's autotuner.
One step = one Maximus call over all users (user quantisation, k-means,
theta_b + CBound, per-cluster lists, the two-pass tensor-core walk, the
exact rescore), replayed from a captured CUDA graph on a created stream,
with users and items already resident in HBM.  The step's value is the
line's `value`.

In the same run, on the same inputs, `legs` times the other forms the
metric compares: the BF16 blocked multiply with fused select (Sec. II-C,
graph replays) and the plain FP32 CUDA-core blocked multiply (plain calls),
each with its users/sec and its own roofline.  `e2e` is the default form
through the host-buffer entry point (pinned host users in, host results
out, copies inside the timed region).  `cpu_baseline` is the FP64 oracle
on a bounded user sample on the host cores; the GPU's results for those
users are compared with the oracle's (`exact_sample`).

Rooflines (every kernel): the slowest of three ceilings -- tensor (or FP32
FMA) FLOPs at the measured peak, HBM bytes at the measured copy bandwidth,
and the select's issue rate at one instruction per score -- over the
kernel's own device time (CUDA events around its launches).

    python bench.py [--gpus N] [--steps K] [--warmup W]
                    [--workload NAME] [--method maximus|bmm|select]
                    [--dtype bf16|fp32] [--f F] [--k K] [--legs bmm,fp32]
                    [--impl ours|reference] [--serve]

Under torchrun (N > 1) the job's user matrix is N x the workload's users;
rank r scores its contiguous slice (weak scaling) with no collective on the
data path; the time is the max over ranks.  --impl reference times the CPU
oracle (FP64 brute force, all host cores) on a bounded user sample per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "kdd-1000000x624961"
METRIC = "exact top-K users/sec (BF16/FP8+rescore & Maximus vs FP32 BMM), % roofline"


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--dtype", default="auto", choices=["auto", "bf16", "fp8", "fp32"])
    p.add_argument("--method", default="maximus", choices=["bmm", "maximus", "select"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--f", type=int, default=0, help="dimension (Netflix shape: 10, 50 or 100; default 50; others: their own f)")
    p.add_argument("--k", type=int, default=10)
    p.add_argument("--clusters", type=int, default=64, help="|C| when the autotuner is off")
    p.add_argument("--no-autotune", action="store_true",
                   help="Maximus / selector: keep --clusters and --block-items instead of mips_autotune")
    p.add_argument("--block-items", type=int, default=0,
                   help="Maximus item block B when the autotuner is off (0: the library default)")
    p.add_argument("--legs", default="bmm,fp32,fp8,arms",
                   help="extra forms timed after the main steps on the same inputs: comma list of bmm (BF16 "
                        "blocked multiply), maximus, fp32 (FP32 CUDA-core blocked multiply), fp8 (the main method on an "
                        "FP8 E4M3 index), arms (the multi-arm selector over BF16, FP8 and FP32 indexes); 'none' for "
                        "none")
    p.add_argument("--leg-steps", type=int, default=3)
    p.add_argument("--users", type=int, default=0,
                   help="use only the first N users (profiling captures; not the benchmark workload)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-graph", action="store_true", help="plain calls instead of captured graphs")
    p.add_argument("--serve", action="store_true",
                   help="serving loop (mips_server_*) on serve-1000000x128: saturated throughput, then Poisson "
                        "arrivals at 0.3 / 0.6 / 0.9 of it with p50 / p99 latency")
    p.add_argument("--kmeans-spherical", action="store_true",
                   help="Maximus / selector: spherical k-means (unit-length centroids)")
    p.add_argument("--fit-frac", type=float, default=0.0,
                   help="Maximus / selector: fit the centroids once on this fraction of the users before the "
                        "warm-up (Sec. III-E dynamic users); timed steps then only assign users")
    return p.parse_args(argv)


from paper_1706_01449_gb300.shard import dist_env, job_throughput, max_over_ranks, rank_users  # noqa: E402


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        sm = [r[0] for r in rows]
        busy = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def kernel_source_hash(names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1706_01449_gb300", "csrc", n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel_key, src_hash):
    """dram bytes per launch of this kernel from the committed ncu summary, if
    it was taken on the same kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != src_hash:
        return None
    return e.get("bytes_per_launch")


def roofline(dtype, f, scores, kernel_ms, hbm_bytes, peaks, peak_src, sm_count, clock_mhz, kernel_key, src_files):
    """The kernel's roofline: the slowest of three ceilings over its device time.

    * tensor (BF16: 2 f FLOP per score at the measured BF16 burst peak;
      FP8 E4M3: at twice it, the nominal FP8 / BF16 ratio) or, for the FP32
      CUDA-core form, FP32 FMA (SMs x 128 FMA/clk x 2 x clock);
    * HBM: the algorithmic bytes at the measured copy bandwidth;
    * select issue: one warp instruction slot per 32 scores on every SM
      sub-partition (SMs x 4 x 32 scores/clk), the algorithmic minimum of
      looking at every score once.
    `frac` is that ceiling's time over the measured time (= achieved / peak
    in the ceiling's own unit)."""
    s = kernel_ms / 1e3
    flops = 2.0 * f * scores
    clk = clock_mhz * 1e6
    ceil = {}
    if dtype == "bf16":
        pk = peaks["bf16_tflops"]
        ceil["tensor"] = {"time_ms": flops / (pk * 1e12) * 1e3, "achieved": flops / s / 1e12, "peak": pk,
                          "unit": "TFLOP/s", "peak_source": f"{peak_src} bf16 burst"}
    elif dtype == "fp8":  # the measured BF16 burst x the nominal FP8 / BF16 ratio (4.5 / 2.25)
        pk = 2.0 * peaks["bf16_tflops"]
        ceil["tensor"] = {"time_ms": flops / (pk * 1e12) * 1e3, "achieved": flops / s / 1e12, "peak": pk,
                          "unit": "TFLOP/s", "peak_source": f"{peak_src} bf16 burst x 2 (nominal fp8 ratio)"}
    else:
        pk = sm_count * 128 * 2 * clk / 1e12
        ceil["alu_fp32_fma"] = {"time_ms": flops / (pk * 1e12) * 1e3, "achieved": flops / s / 1e12, "peak": pk,
                                "unit": "TFLOP/s",
                                "peak_source": f"derived: {sm_count} SMs x 128 FP32 FMA/clk x 2 x {clock_mhz:.0f} MHz"}
    hb = peaks["hbm_gbs"]
    ceil["hbm"] = {"time_ms": hbm_bytes / (hb * 1e9) * 1e3, "achieved": hbm_bytes / s / 1e9, "peak": hb,
                   "unit": "GB/s", "peak_source": f"{peak_src} copy bandwidth"}
    sp = sm_count * 4 * 32 * clk / 1e9
    ceil["select_issue"] = {"time_ms": scores / (sp * 1e9) * 1e3, "achieved": scores / s / 1e9, "peak": sp,
                            "unit": "G scores/s",
                            "peak_source": f"derived: {sm_count} SMs x 4 sub-partitions x 32 lanes x {clock_mhz:.0f} "
                                           f"MHz (one instruction per score)"}
    name = max(ceil, key=lambda k: ceil[k]["time_ms"])
    c = ceil[name]
    bound = {"tensor": "tensor", "hbm": "hbm"}.get(name, "alu")
    return {"bound": bound, "ceiling": name, "achieved": c["achieved"], "peak": c["peak"], "unit": c["unit"],
            "frac": c["achieved"] / c["peak"], "traffic": traffic_for(kernel_key, kernel_source_hash(src_files)),
            "kernel": kernel_key.split()[0], "kernel_ms": kernel_ms, "peak_source": c["peak_source"],
            "algorithmic": {"scores": scores, "flops": flops, "hbm_bytes": hbm_bytes},
            "ceilings_ms": {k: v["time_ms"] for k, v in ceil.items()},
            "fracs": {k: v["time_ms"] / kernel_ms for k, v in ceil.items()}}


def cpu_baseline(U, I, K, target_s=12.0, max_users=20000):
    """The oracle as it stands (FP64 brute force, full sort, OpenMP over all
    host cores) on a bounded user sample; users/sec, plus the oracle's
    results for those users (the first n of the workload)."""
    import oracle
    oracle.build()
    n0 = min(32, U.shape[0])
    t = time.perf_counter()
    _, _, nt = oracle.topk(U[:n0], I, K, return_threads=True)
    per_user = (time.perf_counter() - t) / n0
    n = int(min(max_users, U.shape[0], max(n0, target_s / max(per_user, 1e-9))))
    t = time.perf_counter()
    idx, sc, nt = oracle.topk(U[:n], I, K, return_threads=True)
    dt = time.perf_counter() - t
    return ({"value": n / dt, "unit": "users/s", "cores": nt, "kind": "oracle",
             "sample": f"first {n} users of the workload ({dt:.1f} s of FP64 brute force, full sort per user)"},
            idx, sc)


def cpu_fp32_bmm(U, I, K, target_s=4.0, max_users=200000, block=4096):
    """The plain multithreaded FP32 CPU form: blocked torch.mm on the host
    (all threads) and torch.topk per block of users, on a bounded user
    sample; users/sec.  FP32 and not tie-aware, so not exact: a speed
    reference only.  Blocks are capped so a block's scores stay near 1 GB."""
    import numpy as np
    import torch
    block = max(16, min(block, (1 << 28) // max(1, I.shape[0])))
    It = torch.from_numpy(np.ascontiguousarray(I, dtype=np.float32)).t().contiguous()

    def run(n):
        for u0 in range(0, n, block):
            S = torch.from_numpy(U[u0:min(n, u0 + block)]) @ It
            torch.topk(S, K, dim=1)

    n0 = min(block, U.shape[0])
    t = time.perf_counter()
    run(n0)
    per_user = (time.perf_counter() - t) / n0
    n = int(min(max_users, U.shape[0], max(n0, target_s / max(per_user, 1e-9))))
    t = time.perf_counter()
    run(n)
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": "users/s", "cores": torch.get_num_threads(),
            "kind": "fp32 torch.mm + torch.topk on the host (not exact)",
            "sample": f"first {n} users of the workload in blocks of {block} ({dt:.1f} s)"}


def exact_sample(gpu_idx, gpu_sc, ref_idx, ref_sc):
    """The GPU's rows for the oracle's sample users against the oracle's:
    index equality and the largest score error relative to |oracle score|
    (floor 1e-30)."""
    import numpy as np
    n = ref_idx.shape[0]
    gi, gs = gpu_idx[:n], gpu_sc[:n]
    err = np.abs(gs - ref_sc) / np.maximum(np.abs(ref_sc), 1e-30)
    return {"users": int(n), "indices_equal": bool(np.array_equal(gi, ref_idx)),
            "rows_differing": int((gi != ref_idx).any(axis=1).sum()), "max_rel_score_err": float(err.max())}


def make_inputs(args, rank):
    from paper_1706_01449_gb300 import synth
    W = synth.WORKLOADS[args.workload]
    f = (args.f or W["fs"][1]) if "fs" in W else W["f"]
    n = args.users if getattr(args, "users", 0) else None
    U = rank_users(args.workload, rank, f=f, n=n)
    I = synth.make_items(W, seed=0, f=f)
    return W, f, U, I


def run_reference(args):
    """The oracle as it stands (FP64 brute force, full sort per user, all
    host cores) on a bounded sample of the workload's users per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    _, f, U, I = make_inputs(args, 0)
    K = args.k
    n0 = 32
    t = time.perf_counter()
    _, _, nt = oracle.topk(U[:n0], I, K, return_threads=True)
    per_user = (time.perf_counter() - t) / n0
    n = int(max(n0, min(U.shape[0], 8.0 / max(per_user, 1e-9))))
    for w in range(args.warmup):
        oracle.topk(U[:n], I, K)
    times = []
    for s in range(args.steps):
        lo = (s * n) % max(1, U.shape[0] - n)
        t = time.perf_counter()
        oracle.topk(U[lo:lo + n], I, K)
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    value = n / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "users/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload} f={f} K={K}", "users_per_step": n,
                       "n_items": int(I.shape[0]), "f": f, "K": K, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "users/s", "cores": nt, "kind": "oracle",
                             "sample": f"{n} users per step, FP64 brute force with full sort per user"},
            "e2e": {"value": value, "unit": "users/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Serving loop: requests of 1..4096 users (log-uniform) with K from
    {1, 10, 100}; first all at once (saturated throughput), then Poisson
    arrivals at three fractions of that request rate."""
    import numpy as np
    import torch
    from paper_1706_01449_gb300 import build as libbuild
    from paper_1706_01449_gb300 import mips, synth
    libbuild.build()
    W = synth.WORKLOADS["serve-1000000x128"]
    f = W["f"]
    I = synth.make_items(W, 0)
    index = mips.build_index(torch.from_numpy(I).cuda(), dtype="bf16")
    rng = np.random.default_rng(0)
    offset = [0]

    def make_requests(n):
        out = []
        for _ in range(n):
            m = int(round(np.exp(rng.uniform(0, np.log(4096)))))
            out.append((synth.serving_users(m, f, 1, offset[0]), int(rng.choice(W["ks"]))))
            offset[0] += m
        return out

    srv = mips.Server(index, method="bmm", slots=2, max_batch_users=8192)
    for U, K in make_requests(12):  # warm-up (workspaces, pinned staging)
        srv.wait(srv.submit(U, K))
    reqs = make_requests(96)
    ids = [srv.submit(U, K) for U, K in reqs]
    infos = [srv.wait(i, timeout=600)[2] for i in ids]
    span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
    users = sum(U.shape[0] for U, _ in reqs)
    sat_users, sat_rate = users / span, len(reqs) / span
    loads = {}
    for frac in (0.3, 0.6, 0.9):
        reqs = make_requests(96)
        gaps = rng.exponential(1.0 / (frac * sat_rate), size=len(reqs))
        t0 = time.perf_counter()
        ids, t = [], 0.0
        for (U, K), g in zip(reqs, gaps):
            t += g
            while time.perf_counter() - t0 < t:
                time.sleep(0.0001)
            ids.append(srv.submit(U, K))
        infos = [srv.wait(i, timeout=600)[2] for i in ids]
        lat = np.array([i["t_done"] - i["t_submit"] for i in infos]) * 1e3
        sp = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
        loads[str(frac)] = {"requests_per_s": round(len(reqs) / sp, 1),
                            "users_per_s": sum(U.shape[0] for U, _ in reqs) / sp,
                            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                            "mean_batch_users": float(np.mean([i["batch_users"] for i in infos]))}
    srv.close()
    index.close()
    print(json.dumps({"metric": "serving users/sec (saturated)", "value": sat_users, "unit": "users/s",
                      "n_gpus": 1, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
                      "config": {"workload": "serve-1000000x128", "n_items": W["n_items"], "f": f,
                                 "request_users": "1..4096 log-uniform", "K": list(W["ks"]), "slots": 2,
                                 "max_batch_users": 8192, "requests_per_load": 96},
                      "saturated_requests_per_s": sat_rate, "loads": loads}), flush=True)


def score_roofline(dtype, walked, f, nU, nI, K, stats, peaks, peak_src, sm, clk, workload, walk_cfg=None):
    """Roofline of the call's dominant kernel from its counters: the fused
    score + select kernel (every (user, item) pair), or the Maximus walk
    (the pairs it scored).  Algorithmic bytes: user rows and item rows once
    in the operand dtype, candidate lists out (8 bytes each)."""
    scores = stats["pairs_scored"] if walked else nU * nI
    b = {"bf16": 2, "fp8": 1}.get(dtype, 4)
    hbm = nU * f * b + nI * f * b + 8 * stats["cand_emitted"]
    kms = stats["ms_kernel"] or (stats["ms_walk"] if walked else stats["ms_score"])
    kern = "tc_score_select" if dtype in ("bf16", "fp8") else ("fp32_score_select" if not walked else "maximus_walk")
    key = f"{kern}{' walk' if walked else ''} {dtype} {workload} f={f} K={K}"
    if walked and walk_cfg:  # the walk's traffic depends on |C| and the item block
        key += f" C={walk_cfg[0]} B={walk_cfg[1]}"
    src = (["tc_topk.cu", "tc_ptx.cuh", "tc_topk.h"] if dtype in ("bf16", "fp8")
           else ["fp32_topk.cu" if not walked else "maximus.cu"])
    return roofline(dtype, f, scores, kms, hbm, peaks, peak_src, sm, clk, key, src)


def timed_steps(step, n_warm, n_steps, stream, flush, index, mips):
    """n_warm untimed calls, then n_steps timed ones (CUDA events on the
    call's stream, L2 flushed before each); per-step ms, the dominant
    kernel's ms, kernel launches, and the last step's counters."""
    import torch
    for _ in range(n_warm):
        flush.fill_(1.0)
        step()
    mips.sync(index)
    ms, launches, stats = [], 0, None
    kms = []
    for _ in range(n_steps):
        flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        stats = mips.get_stats(index)
        kms.append(stats["ms_kernel"])
        launches += stats["launches"]
    mips.sync(index)
    return ms, kms, launches, stats


def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    import torch
    from paper_1706_01449_gb300 import build as libbuild
    from paper_1706_01449_gb300 import mips

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(mips.LIB_PATH):
        libbuild.build()
    if world > 1:
        torch.distributed.barrier()
    dev = torch.device("cuda", local)

    W, f, U, I = make_inputs(args, rank)
    K = args.k
    nU, nI = U.shape[0], I.shape[0]
    dtype = args.dtype
    I_d = torch.from_numpy(I).to(dev)
    U_d = torch.from_numpy(U).to(dev)
    index = None
    for cand in (["bf16", "fp32"] if dtype == "auto" else [dtype]):
        try:
            index = mips.build_index(I_d, clusters=args.clusters, dtype=cand, kmeans_spherical=args.kmeans_spherical,
                                     block_items=args.block_items)
            dtype = cand
            break
        except mips.MipsError as e:
            if e.status != mips.MIPS_ERR_UNIMPLEMENTED or cand == "fp32":
                raise
    out_idx = torch.empty((nU, K), dtype=torch.int32, device=dev)
    out_sc = torch.empty((nU, K), dtype=torch.float64, device=dev)
    use_graph = args.method != "select" and not args.no_graph
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)  # torch work (flush, events) and the calls share it
    last_report = {}

    def make_step(idx, method, oi, osc, graph):
        fn = {"bmm": mips.topk, "maximus": mips.topk_maximus}.get(method)

        def step():
            if method == "select":
                last_report.update(mips.select(idx, U_d, K, oi, osc, stream=stream)[2])
            elif graph:
                mips.topk_graph(idx, U_d, K, method, oi, osc, stream=stream)
            else:
                fn(idx, U_d, K, oi, osc, stream=stream)
        return step

    fit = None
    if args.fit_frac > 0 and args.method != "bmm":
        n_fit = max(1, int(round(nU * args.fit_frac)))
        t0 = time.perf_counter()
        mips.fit_clusters(index, U_d[:n_fit], stream=stream)
        mips.sync(index, stream)
        fit = {"users": n_fit, "seconds": time.perf_counter() - t0}
    tune = None
    if not args.no_autotune and args.method != "bmm":
        tune = mips.autotune(index, U_d, K, stream=stream)
        tune = {"clusters": tune["clusters"], "block_items": tune["block_items"],
                "sample_users": tune["sample_users"], "seconds": tune["t_tune"], "candidates": len(tune["tried"])}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    step = make_step(index, args.method, out_idx, out_sc, use_graph)
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    mips.sync(index)

    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms, kern_ms, launches, stats = timed_steps(step, 0, args.steps, stream, flush, index, mips)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()

    total_ms = max_over_ranks(sum(step_ms), device=dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(nU, world, ms_per_step)

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        U_h = torch.from_numpy(U).pin_memory()
        oi_h = torch.empty((nU, K), dtype=torch.int32).pin_memory()
        os_h = torch.empty((nU, K), dtype=torch.float64).pin_memory()
        mips.topk_host(index, U_h, K, args.method, oi_h, os_h)
        ts = []
        for _ in range(min(3, args.steps)):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t = time.perf_counter()
            mips.topk_host(index, U_h, K, args.method, oi_h, os_h)
            ts.append(time.perf_counter() - t)
        e2e_s = max_over_ranks(statistics.median(ts), device=dev)
        e2e = {"value": world * nU / e2e_s, "unit": "users/s",
               "h2d_bytes_per_step": int(U_h.numel() * 4), "d2h_bytes_per_step": int(nU * K * (4 + 8)),
               "entry_point": "mips_topk_host", "same_result_as_device_call":
                   bool(torch.equal(oi_h, out_idx.cpu()) and torch.equal(os_h, out_sc.cpu()))}

    if rank != 0:
        index.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peaks, peak_src = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm = props.multi_processor_count
    clk = float(peaks.get("sm_max_mhz", 2070.0))
    walked = args.method == "maximus" or (args.method == "select" and stats["ms_walk"] > 0 and not stats["ms_score"])
    st_main = dict(stats)
    st_main["ms_kernel"] = statistics.mean(kern_ms) if any(kern_ms) else 0.0
    if args.method == "select":  # the selector's counters are those of its last run (the users outside the sample)
        nU_sel = nU - last_report.get("sample_users", 0)
    else:
        nU_sel = nU
    main_cfg = (stats.get("clusters"), tune["block_items"] if tune else (args.block_items or 4096))
    rl = score_roofline(dtype, walked, f, nU_sel, nI, K, st_main, peaks, peak_src, sm, clk, args.workload, main_cfg)
    rl["launches_per_step"] = 2 if walked else 1

    # the other forms, same inputs, same run (one GPU only)
    legs = {}
    leg_names = [x for x in args.legs.split(",") if x and x != "none"] if world == 1 else []
    for leg in leg_names:
        if leg == args.method and dtype == "bf16":
            continue
        if leg not in ("bmm", "maximus", "fp32", "fp8", "arms"):
            raise SystemExit(f"unknown leg {leg}")
        if leg == "arms":  # the multi-arm selector over BF16, FP8 and FP32 indexes of the same items
            oi = torch.empty_like(out_idx)
            osc = torch.empty_like(out_sc)
            extra = [mips.build_index(I_d, clusters=args.clusters, dtype=d) for d in ("fp8", "fp32")]
            arms_rep = {}

            def astep():
                arms_rep.update(mips.select_arms([index] + extra, U_d, K, 0, oi, osc, stream=stream)[2])
            lms, _, _, _ = timed_steps(astep, 1, args.leg_steps, stream, flush, index, mips)
            names = {0: "fp32", 1: "bf16", 2: "fp8"}
            arms = [{"dtype": names[a["dtype"]], "method": "maximus" if a["method"] else "bmm",
                     "est_ms_all_users": a["est_mean"] * 1e3, "ci95_ms": a["est_ci"] * 1e3, "rounds": a["rounds"],
                     "dropped": bool(a["dropped"])} for a in arms_rep["arms"]]
            legs["arms"] = {"value": nU / (statistics.mean(lms) / 1e3), "unit": "users/s",
                            "ms_per_step": statistics.mean(lms), "steps": args.leg_steps, "warmup": 1,
                            "same_result_as_main": bool(torch.equal(oi, out_idx) and torch.equal(osc, out_sc)),
                            "choice": arms[arms_rep["choice"]], "separated": bool(arms_rep["separated"]),
                            "rounds": arms_rep["rounds"], "sample_users": arms_rep["sample_users"],
                            "overhead_frac": arms_rep["t_sample"] / arms_rep["t_total"], "arms": arms}
            for x in extra:
                x.close()
            del oi, osc
            continue
        oi = torch.empty_like(out_idx)
        osc = torch.empty_like(out_sc)
        if leg == "fp32":
            idx_l = mips.build_index(I_d, clusters=args.clusters, dtype="fp32")
            l_method, l_dtype, l_graph, n_warm = "bmm", "fp32", False, 1
        elif leg == "fp8":  # the main method on an FP8 E4M3 index of the same items
            idx_l = mips.build_index(I_d, clusters=args.clusters, dtype="fp8")
            l_method = "maximus" if args.method == "select" else args.method
            l_dtype, l_graph, n_warm = "fp8", use_graph, 2
        else:
            idx_l = index
            l_method, l_dtype, l_graph, n_warm = leg, dtype, use_graph, 2
        l_block = args.block_items or 4096
        if l_method == "maximus" and leg != "fp32" and not args.no_autotune:
            l_block = mips.autotune(idx_l, U_d, K, stream=stream)["block_items"]
        lstep = make_step(idx_l, l_method, oi, osc, l_graph)
        lms, lkms, _, lst = timed_steps(lstep, n_warm, args.leg_steps, stream, flush, idx_l, mips)
        lst = dict(lst)
        lst["ms_kernel"] = statistics.mean(lkms)
        l_walk = l_method == "maximus"
        lrl = score_roofline(l_dtype, l_walk, f, nU, nI, K, lst, peaks, peak_src, sm, clk, args.workload,
                             (lst.get("clusters"), l_block))
        legs[leg] = {"value": nU / (statistics.mean(lms) / 1e3), "unit": "users/s", "ms_per_step": statistics.mean(lms),
                     "steps": args.leg_steps, "warmup": n_warm, "candidate_pass": l_dtype, "method": l_method,
                     "candidates_per_user": lst.get("cand_emitted", 0) / nU, "rescored_per_user":
                         lst.get("cand_rescored", 0) / nU, "users_overflow": lst.get("users_overflow", 0),
                     "launch": "cuda graph replay" if l_graph else "plain calls",
                     "same_result_as_main": bool(torch.equal(oi, out_idx) and torch.equal(osc, out_sc)),
                     "stages_ms_last_step": {k: lst[k] for k in ("ms_prep", "ms_score", "ms_rescore", "ms_kmeans",
                                                                 "ms_bounds", "ms_sort", "ms_walk", "ms_total")},
                     "roofline": lrl}
        if idx_l is not index:
            idx_l.close()
        del oi, osc

    cpu = cpu32 = exact = None
    if not args.no_cpu_baseline and world == 1:
        cpu, ref_idx, ref_sc = cpu_baseline(U, I, K)
        n_chk = ref_idx.shape[0]
        exact = exact_sample(out_idx[:n_chk].cpu().numpy(), out_sc[:n_chk].cpu().numpy(), ref_idx, ref_sc)
        cpu32 = cpu_fp32_bmm(U, I, K)

    tiles = (stats["blocks_walked"] if walked else ((nU_sel + 127) // 128) * ((nI + 255) // 256))
    line = {
        "metric": METRIC, "value": value, "unit": "users/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"bf16": "bf16", "fp8": "fp8_e4m3"}.get(dtype, "f32"),
        "data": "synthetic",
        "config": {"workload": f"{args.workload} f={f} K={K}" + (f" first {nU} users" if args.users else ""),
                   "n_users": nU, "n_items": nI, "f": f, "K": K,
                   "method": args.method, "candidate_pass": dtype, "rescore": "compensated fp32 + fp64 tie check",
                   "launch": "cuda graph replay" if use_graph else "plain calls",
                   **({"clusters": stats["clusters"]} if args.method != "bmm" else {}),
                   **({"autotune": tune} if tune else {}),
                   **({"centroids_fitted_before_timing": fit} if fit else {}),
                   **({"kmeans": "spherical"} if args.kmeans_spherical else {}),
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"users sharded: {world} rank(s), contiguous slices of one user matrix"},
        "roofline": rl,
        "legs": legs,
        "cpu_baseline": cpu,
        "cpu_fp32_bmm": cpu32,
        "exact_sample": exact,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "stages_ms_last_step": {k: stats[k] for k in ("ms_prep", "ms_score", "ms_rescore", "ms_kmeans",
                                                       "ms_bounds", "ms_sort", "ms_walk", "ms_total", "ms_kernel")},
        "candidates_per_user": stats["cand_emitted"] / nU, "rescored_per_user": stats["cand_rescored"] / nU,
        "users_overflow": stats["users_overflow"], "users_fp64": stats["users_fp64"],
        **({"pairs_scored_per_user": stats["pairs_scored"] / nU} if walked else {}),
        # per warp and 64-score chunk of the tiles the score kernel processed
        # (128 users x 256 items each, eight select warps of 128 columns)
        "select_slow_chunk_frac": (stats["select_slow"] / (tiles * 8 * 2) if dtype == "bf16" and tiles else None),
    }
    print(json.dumps(line), flush=True)
    index.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
