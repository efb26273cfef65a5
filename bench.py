"""Benchmark: exact batch top-K MIPS throughput (users/sec) on GB300.

One step = one mips_topk call (the whole hot path: user quantisation,
fused score + select, exact rescore) over all users of the workload, with
users and items already resident in HBM.  Prints ONE JSON line (rank 0).
The blocked multiply and Maximus steps go through mips_topk_graph on a
created stream (the call is captured into a CUDA graph in the warm-up and
replayed); --no-graph runs the plain calls.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype bf16|fp32]
                    [--method bmm|maximus|select] [--f 50] [--k 10]
                    [--impl ours|reference] [--no-graph]

Under torchrun (N > 1) every rank runs the same workload on its own users
(seed = rank) with no collective on the data path: weak scaling; the time
is the max over ranks.  --impl reference times the CPU oracle (FP64 brute
force, all host cores) on a bounded user sample per step.
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

WORKLOAD = "netflix-480189x17770"
SM_COUNT_FALLBACK = 152


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--dtype", default="auto", choices=["auto", "bf16", "fp32"])
    p.add_argument("--method", default="bmm", choices=["bmm", "maximus", "select"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--f", type=int, default=50)
    p.add_argument("--k", type=int, default=10)
    p.add_argument("--clusters", type=int, default=64)
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
                        "warm-up (Sec. IV-E dynamic users); timed steps then only assign users")
    p.add_argument("--autotune", action="store_true",
                   help="Maximus / selector: pick |C| and B with mips_autotune before the warm-up (timed separately)")
    return p.parse_args()


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


def cpu_baseline(U, I, K, target_s=12.0, max_users=20000):
    """The oracle as it stands (FP64 brute force, full sort, OpenMP over all
    host cores) on a bounded user sample; users/sec."""
    import oracle
    oracle.build()
    n0 = min(64, U.shape[0])
    t = time.perf_counter()
    _, _, nt = oracle.topk(U[:n0], I, K, return_threads=True)
    per_user = (time.perf_counter() - t) / n0
    n = int(min(max_users, U.shape[0], max(n0, target_s / max(per_user, 1e-9))))
    t = time.perf_counter()
    _, _, nt = oracle.topk(U[:n], I, K, return_threads=True)
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": "users/s", "cores": nt, "kind": "oracle",
            "sample": f"first {n} users of the workload ({dt:.1f} s of FP64 brute force, full sort per user)"}


def cpu_fp32_bmm(U, I, K, target_s=4.0, max_users=200000, block=4096):
    """The plain multithreaded FP32 CPU form: blocked torch.mm on the host
    (all threads) and torch.topk per block of users, on a bounded user
    sample; users/sec.  FP32 and not tie-aware, so not exact: a speed
    reference only."""
    import numpy as np
    import torch
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


def make_inputs(args, rank):
    from paper_1706_01449_gb300 import synth
    W = synth.WORKLOADS[args.workload]
    f = args.f if "fs" in W else W["f"]
    n = args.users if getattr(args, "users", 0) else None
    U = rank_users(args.workload, rank, f=f, n=n)
    I = synth.make_items(W, seed=0, f=f)
    return W, f, U, I


def run_reference(args):
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
    line = {"impl": "reference", "metric": "exact top-K users/sec", "value": value, "unit": "users/s",
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


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    import numpy as np
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
            index = mips.build_index(I_d, clusters=args.clusters, dtype=cand, kmeans_spherical=args.kmeans_spherical)
            dtype = cand
            break
        except mips.MipsError as e:
            if e.status != mips.MIPS_ERR_UNIMPLEMENTED or cand == "fp32":
                raise
    out_idx = torch.empty((nU, K), dtype=torch.int32, device=dev)
    out_sc = torch.empty((nU, K), dtype=torch.float64, device=dev)
    fn = {"bmm": mips.topk, "maximus": mips.topk_maximus}.get(args.method)
    use_graph = args.method != "select" and not args.no_graph
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)  # torch work (flush, events) and the calls share it

    last_report = {}

    def step():
        if args.method == "select":
            last_report.update(mips.select(index, U_d, K, out_idx, out_sc, stream=stream)[2])
        elif use_graph:
            mips.topk_graph(index, U_d, K, args.method, out_idx, out_sc, stream=stream)
        else:
            fn(index, U_d, K, out_idx, out_sc, stream=stream)

    fit = None
    if args.fit_frac > 0 and args.method != "bmm":
        n_fit = max(1, int(round(nU * args.fit_frac)))
        t0 = time.perf_counter()
        mips.fit_clusters(index, U_d[:n_fit], stream=stream)
        mips.sync(index, stream)
        fit = {"users": n_fit, "seconds": time.perf_counter() - t0}
    tune = None
    if args.autotune and args.method != "bmm":
        tune = mips.autotune(index, U_d, K, stream=stream)
        tune = {"clusters": tune["clusters"], "block_items": tune["block_items"],
                "sample_users": tune["sample_users"], "seconds": tune["t_tune"], "candidates": len(tune["tried"])}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    mips.sync(index)

    sampler = ClockSampler(local)
    sampler.start()
    step_ms, score_ms, launches = [], [], 0
    stats = None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stats = mips.get_stats(index)
        score_ms.append(stats["ms_score"] if args.method == "bmm" else stats["ms_walk"] or stats["ms_score"])
        launches += stats["launches"]
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    mips.sync(index)

    total_ms = max_over_ranks(sum(step_ms), device=dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(nU, world, ms_per_step)

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        U_h = torch.from_numpy(U).pin_memory()
        oi_h = torch.empty((nU, K), dtype=torch.int32).pin_memory()
        os_h = torch.empty((nU, K), dtype=torch.float64).pin_memory()
        method = {"bmm": "bmm", "maximus": "maximus", "select": "select"}[args.method]
        mips.topk_host(index, U_h, K, method, oi_h, os_h)
        ts = []
        for _ in range(min(3, args.steps)):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t = time.perf_counter()
            mips.topk_host(index, U_h, K, method, oi_h, os_h)
            ts.append(time.perf_counter() - t)
        e2e = {"value": nU / statistics.median(ts), "unit": "users/s",
               "h2d_bytes_per_step": int(U_h.numel() * 4), "d2h_bytes_per_step": int(nU * K * (4 + 8))}

    if rank != 0:
        index.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peaks, peak_src = load_peaks()
    # algorithmic work of the scoring kernel: every (user, item) pair it
    # scores; the Maximus walk scores only the pairs its bounds leave
    walked = args.method == "maximus" or (args.method == "select" and stats["ms_walk"] > 0 and not stats["ms_score"])
    # (the selector's stage times are those of its last run: the users
    # outside the timed sample)
    scored_users = nU - last_report.get("sample_users", 0) if args.method == "select" else nU
    flops = 2.0 * f * (stats["pairs_scored"] if walked else scored_users * nI)
    kms = statistics.mean(score_ms)
    if dtype == "bf16":
        bound, peak, unit = "tensor", peaks["bf16_tflops"], "TFLOP/s"
        kernel_key = f"tc_score_select bf16 {args.workload} f={f} K={K}"
        src = ["tc_topk.cu"]
    else:
        props = torch.cuda.get_device_properties(dev)
        sm = getattr(props, "multi_processor_count", SM_COUNT_FALLBACK)
        bound, unit = "alu", "TFLOP/s"
        peak = sm * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        kernel_key = f"fp32_score_select {args.workload} f={f} K={K}"
        src = ["fp32_topk.cu"]
    achieved = flops / (kms / 1e3) / 1e12
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": traffic_for(kernel_key, kernel_source_hash(src)),
                "kernel": kernel_key.split()[0], "kernel_ms": kms,
                "peak_source": (f"{peak_src} bf16 burst" if bound == "tensor"
                                else f"derived: SMs x 128 FP32 FMA/clk x 2 x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz"),
                "algorithmic_flops_per_launch": flops}

    cpu = cpu32 = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(U, I, K)
        cpu32 = cpu_fp32_bmm(U, I, K)

    tiles = (stats["blocks_walked"] if walked else ((nU + 127) // 128) * ((nI + 255) // 256))
    line = {
        "metric": "exact top-K users/sec", "value": value, "unit": "users/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if dtype == "bf16" else "f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} f={f} K={K}" + (f" first {nU} users" if args.users else ""),
                   "n_users": nU, "n_items": nI, "f": f, "K": K,
                   "method": args.method, "candidate_pass": dtype, "rescore": "compensated fp32 + fp64 tie check",
                   "launch": "cuda graph replay" if use_graph else "plain calls",
                   **({"clusters": stats["clusters"]} if args.method != "bmm" else {}),
                   **({"autotune": tune} if tune else {}),
                   **({"centroids_fitted_before_timing": fit} if fit else {}),
                   **({"kmeans": "spherical"} if args.kmeans_spherical else {}),
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"users sharded, {world} rank(s)"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cpu_fp32_bmm": cpu32,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "stages_ms_last_step": {k: stats[k] for k in ("ms_prep", "ms_score", "ms_rescore", "ms_kmeans",
                                                       "ms_bounds", "ms_sort", "ms_walk", "ms_total")},
        "candidates_per_user": stats["cand_emitted"] / nU, "rescored_per_user": stats["cand_rescored"] / nU,
        "users_overflow": stats["users_overflow"], "users_fp64": stats["users_fp64"],
        **({"pairs_scored_per_user": stats["pairs_scored"] / nU} if walked else {}),
        # per warp and 16-score chunk of the tiles the score kernel processed
        # (128 users x 256 items each)
        "select_slow_chunk_frac": (stats["select_slow"] / (tiles * 8 * 8) if dtype == "bf16" and tiles else None),
    }
    print(json.dumps(line), flush=True)
    index.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
