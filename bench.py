#!/usr/bin/env python
"""Throughput benchmark of the GB300 sampled-dominator-tree estimator.

A step is one AdvancedGreedy query (Alg. 3): b rounds, each one Alg. 2 call over theta sampled
graphs (live-edge decisions, BFS from the seeds, dominator tree, subtree sizes, counter
update) followed by the blocker selection. Workload: R-MAT n=2^17, m=2^20 (a,b,c,d =
.57/.19/.19/.05), weighted-cascade thresholds, |S|=50 uniform seeds, b=50, theta=10^5.

value = sampled graphs processed per second (b * theta per step) with the graph and the seed
set already on the device; e2e = the same metric through the C ABI from pinned host buffers,
graph upload and blocker read-back included in every step.

Under torchrun (N > 1) every rank runs an independent query replica on its own GPU (the path
has no exchange step); value = samples of all ranks / the slowest rank's time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "samples/s batched vs one-query-per-launch (bit-exact); AG/GR wall time; p99"
WORKLOAD = "rmat17-wc-advanced-greedy"
L2_FLUSH_BYTES = 512 << 20
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--ref-step-seconds", type=float, default=10.0,
                   help="--impl reference: target host time of one step (a bounded sample)")
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="target CPU time of the oracle baseline sample")
    p.add_argument("--workload", choices=("rmat17", "batch256", "serving", "rmat22"), default="rmat17",
                   help="rmat17: one AdvancedGreedy query on R-MAT 2^17 (the headline line); "
                        "batch256: 256 Chung-Lu/TR queries, batched vs one query per launch; "
                        "serving: Poisson request stream on the R-MAT 2^17 and 2^22 graphs; "
                        "rmat22: AG and GR wall time of the large single query (R-MAT 2^22)")
    p.add_argument("--requests", type=int, default=30,
                   help="serving: number of requests (the full configuration has 2,000)")
    p.add_argument("--b", type=int, default=None,
                   help="rmat22: budget override (smaller cases for profiling; default 200)")
    p.add_argument("--theta", type=int, default=None,
                   help="rmat22: samples per round override (default 2*10^5)")
    return p.parse_args(argv)


# --------------------------------------------------------------------------------------------
# ranks and aggregation
# --------------------------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def aggregate(local_seconds: float, local_units: float, world: int, reduce_max=None,
              reduce_sum=None):
    """Whole-job throughput: units of all ranks / slowest rank's time (max over ranks)."""
    t = reduce_max(local_seconds) if reduce_max else local_seconds
    u = reduce_sum(local_units) if reduce_sum else local_units * world
    return u / t if t > 0 else 0.0, t


def make_reducers(dist):
    if dist is None:
        return None, None
    import torch

    def red(x, op):
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=op)
        return float(t.item())

    return (lambda x: red(x, dist.ReduceOp.MAX)), (lambda x: red(x, dist.ReduceOp.SUM))


# --------------------------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="imin_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.path is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(REASONS, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------------------------------
# roofline accounting
# --------------------------------------------------------------------------------------------

def algorithmic_bytes(stats: dict, tier: int, n_seeds: int) -> float:
    """Bytes the method must move for the samples finished by one kernel tier:
    8|R| (row offsets of every reached vertex) + 4 E_R (threshold of every examined edge)
    + 4 L (target of every live edge) + 8 |R \\ S| (one uint64 counter per reached non-seed)."""
    r = stats["tier_reached"][tier]
    e = stats["tier_examined_edges"][tier]
    l_ = stats["tier_live_edges"][tier]
    s = stats["tier_samples"][tier] * n_seeds
    return 8.0 * r + 4.0 * e + 4.0 * l_ + 8.0 * (r - s)


KERNEL_SOURCES = ("sample_cta.cu", "sample_cta.cuh", "imin_dev.cuh", "internal.h")


def kernel_source_hash() -> str:
    """Hash of the sources that define the block-tier kernel (its translation unit and headers)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2302_13529_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken on the
    current kernel sources (profiles/<kernel>_<workload>.md: 'source_hash:' and
    'dram_bytes_per_launch:' lines); None otherwise."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{WORKLOAD}.md")
    if not os.path.exists(path):
        return None
    src, val = None, None
    for line in open(path):
        if line.startswith("source_hash:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            val = float(line.split(":", 1)[1].strip())
    return val if src == kernel_source_hash() else None


# --------------------------------------------------------------------------------------------
# arms
# --------------------------------------------------------------------------------------------

def cpu_baseline(q, seconds: float):
    """The oracle as it stands (single-threaded C), on a bounded sample of the workload:
    the first `count` sampled graphs of round 0, sized to take about `seconds`."""
    from oracle import oracle as O

    O.lib()
    t = time.perf_counter()
    O.decrease(q.graph, q.seeds, [], 200, q.key, 0)
    per = (time.perf_counter() - t) / 200
    count = int(max(200, min(q.theta, seconds / max(per, 1e-7))))
    t = time.perf_counter()
    O.decrease(q.graph, q.seeds, [], count, q.key, 0)
    dt = time.perf_counter() - t
    return {"value": count / dt, "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": f"round 0, samples 0..{count - 1} of theta={q.theta} ({dt:.1f} s)"}


def run_reference(args, q, rank):
    """The oracle timed on the host cores on the same workload, metric and unit; each step is a
    bounded sample (a range of sampled graphs of one round)."""
    from oracle import oracle as O

    if rank != 0:
        return
    O.lib()
    t = time.perf_counter()
    O.decrease(q.graph, q.seeds, [], 100, q.key, 0)
    per = (time.perf_counter() - t) / 100
    per_step = int(max(100, min(q.theta, args.ref_step_seconds / max(per, 1e-7))))
    for w in range(args.warmup):
        O.decrease(q.graph, q.seeds, [], min(per_step, 200), q.key, w)
    times = []
    for k in range(args.steps):
        t = time.perf_counter()
        O.decrease(q.graph, q.seeds, [], per_step, q.key, k, (k * per_step) % q.theta)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = per_step * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "uint32", "data": "synthetic",
            "config": config_of(q),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} sampled graphs of one round per step"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(q):
    return {"workload": WORKLOAD, "graph": "R-MAT scale 17, m=2^20, (0.57,0.19,0.19,0.05), WC",
            "n": q.graph.n, "m": q.graph.m, "seeds": int(len(q.seeds)), "b": q.b,
            "theta": q.theta, "samples_per_step": q.b * q.theta,
            "l2": "flushed between steps (512 MiB write outside the step events)"}


def run_batch(args, rank, world, dist):
    """256 independent AdvancedGreedy queries (Chung-Lu, n log-uniform in [1e3, 2e5], mean degree
    U[5,20], TR probabilities, |S| U[5,100], b=20, theta=2e4): one batched call (a step) vs the
    same queries one imin_advanced_greedy call at a time; the results must be identical."""
    import numpy as np
    import torch
    from paper_2302_13529_gb300 import build, imin, workloads as W

    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    qs = W.batch_queries(256)
    gen_s = time.perf_counter() - t0
    hs = [imin.load_graph(q.graph) for q in qs]
    items = [(h, q.seeds, q.b, q.theta, q.key + rank) for h, q in zip(hs, qs)]
    samples = sum(q.b * q.theta for q in qs)  # every query runs b rounds (n - |S| >= b here)
    for _ in range(max(args.warmup, 3) if args.warmup else 1):
        imin.batch_advanced_greedy(items)
    torch.cuda.synchronize()
    imin.profile_read(reset=True)
    imin.profile_enable(True)
    launches0 = imin.launch_count()
    times = []
    res = None
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = imin.batch_advanced_greedy(items)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    launches = imin.launch_count() - launches0
    imin.profile_enable(False)
    prof = imin.profile_read(reset=True)
    st = imin.last_stats()
    for h, q in zip(hs, qs):  # the plain calls' per-graph cutoff tuning stays out of their timing
        imin.autotune(h, q.seeds, q.key + rank)
    torch.cuda.synchronize()
    t = time.perf_counter()
    plain = [imin.advanced_greedy(*it) for it in items]
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t
    same = all(np.array_equal(a, b) for a, b in zip(res, plain))
    batched_s = sum(times) / len(times)
    line = {"metric": METRIC, "value": samples / batched_s, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * batched_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "uint32",
            "data": "synthetic",
            "config": {"workload": "batch256-chunglu-tr-advanced-greedy", "queries": len(qs),
                       "b": 20, "theta": 20000, "samples_per_step": samples,
                       "total_edges": int(sum(q.graph.m for q in qs)),
                       "generation_s": round(gen_s, 1)},
            "one_query_per_launch": {"value": samples / plain_s, "unit": "samples/s",
                                     "seconds": plain_s,
                                     "cutoff": "autotuned per graph before timing"},
            "batched_cutoff": int(os.environ.get("IMIN_TIER0_VERTICES", "96") or 96),
            "batched_over_plain": plain_s / batched_s, "bit_exact_vs_plain": same,
            "gpu_launches": launches,
            "kernel_ms": {k: round(v["ms"], 3) for k, v in prof.items()},
            "work": {"reached_per_sample": st["reached"] / max(st["samples"], 1),
                     "examined_edges_per_sample": st["examined_edges"] / max(st["samples"], 1)}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_rmat22(args, rank, world):
    """The large single query: R-MAT n=2^22, m=2^26, WC, |S|=200, b=200, theta=2*10^5, rounds
    captured in one CUDA graph. One AdvancedGreedy query is the step (4*10^7 sampled graphs);
    the warm-up is one 2-round query (module load, cutoff tuning, allocator pools). GreedyReplace
    is timed once after it. Inputs are resident on the device."""
    import torch
    from paper_2302_13529_gb300 import build, imin, workloads as W

    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    q = W.rmat22_query()
    if args.b is not None or args.theta is not None:
        q = W.Query(q.graph, q.seeds, args.b if args.b is not None else q.b,
                    args.theta if args.theta is not None else q.theta, q.key)
    gen_s = time.perf_counter() - t0
    key = q.key + rank
    gh = imin.load_graph(q.graph)
    seeds_d = torch.from_numpy(q.seeds).cuda()
    out_d = torch.empty(q.b, dtype=torch.int32, device="cuda")
    forced = os.environ.get("IMIN_TIER0_VERTICES", "")
    cutoff = int(forced) if forced else imin.autotune(gh, q.seeds, key)
    imin.advanced_greedy(gh, seeds_d, 2, q.theta, key, out=out_d)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    walls = {}
    for name, fn in (("ag", imin.advanced_greedy), ("gr", imin.greedy_replace)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(gh, seeds_d, q.b, q.theta, key, out=out_d)
        e1.record(stream)
        torch.cuda.synchronize()
        walls[name] = e0.elapsed_time(e1) / 1e3
        walls[name + "_stats"] = imin.last_stats()
    st = walls["ag_stats"]
    samples = st["samples"]
    line = {"metric": METRIC, "value": samples / walls["ag"], "unit": "samples/s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": 1e3 * walls["ag"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "uint32", "data": "synthetic",
            "config": {"workload": "rmat22-wc-advanced-greedy", "n": q.graph.n, "m": q.graph.m,
                       "seeds": len(q.seeds), "b": q.b, "theta": q.theta,
                       "warp_block_cutoff": cutoff, "generation_s": round(gen_s, 1),
                       "l2": "graph (528 MB) larger than L2"},
            "ag_wall_s": walls["ag"], "gr_wall_s": walls["gr"],
            "gr_samples": walls["gr_stats"]["samples"],
            "work": {"reached_per_sample": st["reached"] / samples,
                     "examined_edges_per_sample": st["examined_edges"] / samples,
                     "tier_samples": st["tier_samples"]}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serving(args, rank, world):
    """Requests against the R-MAT 2^17 (m=2^20) and R-MAT 2^22 (m=2^26) WC graphs held resident:
    each picks a graph with probability 1/2, |S| ~ U[10, 500], b ~ U[10, 100],
    theta ~ U[1e4, 1e5] (AdvancedGreedy). Phase 1 submits all requests at once to measure the
    saturation rate; phase 2 replays them with Poisson arrivals at 80 % of that rate and reports
    p50/p99 latency and throughput; the serial baseline runs a subset one query at a time."""
    import threading

    import numpy as np
    import torch
    from paper_2302_13529_gb300 import build, imin, workloads as W

    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    g17 = W.rmat17_query().graph
    g22 = W.rmat22_query().graph
    graphs = [g17, g22]
    hs = [imin.load_graph(g) for g in graphs]
    rng = np.random.default_rng(5000 + rank)
    reqs = []
    for i in range(args.requests):
        gi = int(rng.integers(0, 2))
        k = int(rng.integers(10, 501))
        reqs.append((gi, W.uniform_seeds(graphs[gi].n, k, int(rng.integers(1 << 30))),
                     int(rng.integers(10, 101)), int(rng.integers(10_000, 100_001)),
                     int(rng.integers(1 << 62))))
    samples = sum(b * t for _, _, b, t, _ in reqs)

    def serve(arrivals):
        """Submit reqs[:len(arrivals)] at the given offsets (s); return (elapsed, latencies, stats)."""
        todo = reqs[:len(arrivals)]
        lat = [None] * len(todo)
        with imin.Server() as srv:
            t0 = time.perf_counter()
            tickets = [None] * len(todo)

            def submitter():
                for i, (gi, s, b, t, k) in enumerate(todo):
                    wait = arrivals[i] - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(wait)
                    tickets[i] = srv.submit(0, hs[gi], s, b, t, k)

            th = threading.Thread(target=submitter)
            th.start()
            th.join()
            for i, (gi, s, b, t, k) in enumerate(todo):
                _, lat[i] = srv.wait(tickets[i], capacity=b)
            elapsed = time.perf_counter() - t0
            st = srv.stats()
        return elapsed, np.array(lat), st

    serve([0.0] * min(len(reqs), 2))  # warm-up (module load, first plans)
    burst_s, burst_lat, _ = serve([0.0] * len(reqs))
    rate = 0.8 * len(reqs) / burst_s  # requests per second at 80 % of saturation
    gaps = np.random.default_rng(6000 + rank).exponential(1.0 / rate, size=len(reqs))
    poisson_s, lat, st = serve(list(np.cumsum(gaps) - gaps[0]))
    # serial baseline: one query at a time on a subset (about a third of the requests)
    sub_ids = list(range(0, len(reqs), 3))
    t = time.perf_counter()
    for i in sub_ids:
        gi, s, b, th_, k = reqs[i]
        imin.advanced_greedy(hs[gi], s, b, th_, k)
    torch.cuda.synchronize()
    serial_s = time.perf_counter() - t
    serial_samples = sum(reqs[i][2] * reqs[i][3] for i in sub_ids)
    line = {"metric": METRIC, "value": samples / poisson_s, "unit": "samples/s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": 1e3 * poisson_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "uint32", "data": "synthetic",
            "config": {"workload": "serving-rmat17-rmat22-advanced-greedy",
                       "requests": len(reqs), "full_configuration_requests": 2000,
                       "arrivals": f"Poisson at 80% of the burst rate ({rate:.3f} req/s)",
                       "samples": samples},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "burst": {"seconds": burst_s, "samples_per_s": samples / burst_s,
                      "p50_ms": float(np.percentile(burst_lat, 50)),
                      "p99_ms": float(np.percentile(burst_lat, 99))},
            "serial_one_query_at_a_time": {"value": serial_samples / serial_s, "unit": "samples/s",
                                           "requests": len(sub_ids)},
            "server": st}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
    rank, world, local_rank = dist_env()
    from paper_2302_13529_gb300 import workloads as W

    dist = None
    if world > 1:
        import torch.distributed as tdist
        import torch
        if args.impl == "ours" and torch.cuda.is_available():
            torch.cuda.set_device(local_rank)
            tdist.init_process_group("nccl")
        else:
            tdist.init_process_group("gloo")
        dist = tdist

    if args.workload == "batch256":
        run_batch(args, rank, world, dist)
        return
    if args.workload == "serving":
        run_serving(args, rank, world)
        return
    if args.workload == "rmat22":
        run_rmat22(args, rank, world)
        return
    q = W.rmat17_query()
    if args.impl == "reference":
        run_reference(args, q, rank)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    import numpy as np
    import torch
    from paper_2302_13529_gb300 import build, imin

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    key = q.key + rank  # independent replica per rank
    gh = imin.load_graph(q.graph)
    seeds_d = torch.from_numpy(q.seeds).to(dev)
    out_d = torch.empty(q.b, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        imin.advanced_greedy(gh, seeds_d, q.b, q.theta, key, out=out_d)

    # the warp/block cutoff the steps will use (IMIN_TIER0_VERTICES fixes it, e.g. for profiling)
    forced = os.environ.get("IMIN_TIER0_VERTICES", "")
    cutoff = int(forced) if forced else imin.autotune(gh, q.seeds, key)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    reduce_max, reduce_sum = make_reducers(dist)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    imin.profile_read(reset=True)
    imin.profile_enable(True)
    stats_sum = None
    launches0 = imin.launch_count()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[0])
                      if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit()
                      else local_rank) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            step()
            stops[k].record(stream)
            st = imin.last_stats()
            if stats_sum is None:
                stats_sum = st
            else:
                for kk, vv in st.items():
                    stats_sum[kk] = ([a + b for a, b in zip(stats_sum[kk], vv)]
                                     if isinstance(vv, list) else stats_sum[kk] + vv)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = imin.launch_count() - launches0
    imin.profile_enable(False)
    prof = imin.profile_read(reset=True)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, stops)]
    local_s = sum(step_ms) / 1e3
    samples_local = q.b * q.theta * args.steps
    value, slowest = aggregate(local_s, samples_local, world, reduce_max, reduce_sum)
    ms_per_step = 1e3 * slowest / args.steps

    # roofline of the dominant kernel (the sample tier with the most device time)
    tiers = [("sample_tier0", 0), ("sample_tier1", 1), ("sample_tier2", 2), ("sample_cta", 3)]
    kname, tier = max(tiers, key=lambda kt: prof[kt[0]]["ms"])
    kp = prof[kname]
    avg_ms = kp["ms"] / max(kp["launches"], 1)
    alg_bytes = algorithmic_bytes(stats_sum, tier, len(q.seeds)) / max(kp["launches"], 1)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    kfn = "k_sample_cta" if tier == 3 else f"k_sample_tier{tier}"
    traffic = ncu_traffic(kfn)
    total_ms = sum(v["ms"] for v in prof.values())
    roofline = {"kernel": kfn, "bound": "hbm", "achieved": achieved,
                "peak": peak, "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "algorithmic_bytes_per_launch": alg_bytes,
                "avg_launch_ms": avg_ms, "share_of_device_time": kp["ms"] / max(total_ms, 1e-9),
                "kernel_ms": {k: round(v["ms"], 3) for k, v in prof.items()}}

    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "uint32",
            "data": "synthetic", "config": dict(config_of(q), warp_block_cutoff=cutoff),
            "roofline": roofline, "gpu_launches": launches,
            "work": {"reached_per_sample": stats_sum["reached"] / stats_sum["samples"],
                     "examined_edges_per_sample": stats_sum["examined_edges"] / stats_sum["samples"],
                     "live_edges_per_sample": stats_sum["live_edges"] / stats_sum["samples"],
                     "live_edges_per_s": value * stats_sum["live_edges"] / stats_sum["samples"],
                     "tier_samples": stats_sum["tier_samples"]},
            "ag_wall_s": ms_per_step / 1e3}
    clocks = clk.summary()
    if clocks is not None:
        line["clocks"] = clocks

    # GreedyReplace wall time (one query, device-resident inputs)
    ag_blockers = out_d.cpu().numpy().copy()
    torch.cuda.synchronize()
    t = time.perf_counter()
    imin.greedy_replace(gh, seeds_d, q.b, q.theta, key, out=out_d)
    torch.cuda.synchronize()
    line["gr_wall_s"] = time.perf_counter() - t
    gr_blockers = out_d.cpu().numpy().copy()

    # quality of the blocker sets: expected spread by simulation (Def. 3), 10^5 sampled graphs
    # on an independent key, as the paper evaluates its results
    ev_key, ev_theta = (key ^ 0x5EED5EED5EED) & ((1 << 64) - 1), 100_000
    line["expected_spread"] = {
        "theta": ev_theta,
        "no_blockers": imin.estimate_spread(gh, q.seeds, [], ev_theta, ev_key) / ev_theta,
        "advanced_greedy": imin.estimate_spread(gh, q.seeds, ag_blockers, ev_theta, ev_key) / ev_theta,
        "greedy_replace": imin.estimate_spread(gh, q.seeds, gr_blockers, ev_theta, ev_key) / ev_theta}

    # end to end through the C ABI from pinned host buffers
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        rp_h, col_h, thr_h = pin(q.graph.row_ptr), pin(q.graph.col), pin(q.graph.thr.view(np.int32))
        seeds_h = pin(q.seeds)
        out_h = torch.empty(q.b, dtype=torch.int32).pin_memory()
        h2d = rp_h.numel() * 4 + col_h.numel() * 4 + thr_h.numel() * 4 + seeds_h.numel() * 4
        d2h = out_h.numel() * 4
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(e2e_steps):
            g2 = imin.GraphHandle(q.graph.n, rp_h, col_h, thr_h.view(torch.uint32))
            imin.advanced_greedy(g2, seeds_h, q.b, q.theta, key, out=out_h)
            g2.close()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t
        e2e_value, _ = aggregate(e2e_s, q.b * q.theta * e2e_steps, world, reduce_max, reduce_sum)
        line["e2e"] = {"value": e2e_value, "unit": "samples/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                       "includes": "graph upload + validation, warp/block cutoff tuning of the "
                                   "new graph handle, seed upload, 50 rounds, blocker read-back"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(q, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
