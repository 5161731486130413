#!/usr/bin/env python
"""Throughput benchmark of the GB300 sampled-dominator-tree estimator.

Headline (value): a step is one AdvancedGreedy query (Alg. 3) on the mid-scale workload -- R-MAT
n=2^17, m=2^20 (a,b,c,d = .57/.19/.19/.05), weighted-cascade thresholds, |S|=50 uniform seeds,
b=50, theta=10^5: b rounds, each one Alg. 2 call over theta sampled graphs (live-edge decisions,
BFS from the seeds, dominator tree, subtree sizes, counter update) followed by the blocker
selection, all rounds in one captured CUDA graph (the production path). value = sampled graphs
per second with the graph and seeds already on the device; e2e = the same metric through the C
ABI from pinned host buffers, graph upload and blocker read-back included in every step.

The same line carries the metric's other quantities, each measured in this run (N = 1 only):
  batched_vs_plain  256 Chung-Lu TR queries in one batched call vs one call per query
                    (samples/s of both, their ratio, bit-exactness of every result);
  large_query       R-MAT n=2^22, m=2^26, |S|=200, b=200, theta=2*10^5: AG and GR wall time;
  serving           a Poisson request stream on the R-MAT 2^17 and 2^22 graphs: p50/p99 latency
                    and samples/s against serving the same requests one at a time;
  quality           the paper's quality studies on synthetic stand-ins: GreedyReplace's expected
                    spread and time for theta in {10^3, 10^4, 10^5}; Exact vs GreedyReplace on
                    100-vertex graphs (b = 1..3); BaselineGreedy (Alg. 1) vs AdvancedGreedy and
                    GreedyReplace time at b = 10.

Under torchrun (N > 1) every rank runs an independent replica of the headline query on its own
GPU (the path has no exchange step); value = samples of all ranks / the slowest rank's time.
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
SAMPLE_KINDS = (("sample_tier0", 0, "k_sample_tier0"), ("sample_tier1", 1, "k_sample_tier1"),
                ("sample_tier2", 2, "k_sample_tier2"), ("sample_cta", 3, "k_sample_cta"))


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="headline only: skip the batched, large-query and serving legs")
    p.add_argument("--ref-step-seconds", type=float, default=10.0,
                   help="--impl reference: target host time of one step (a bounded sample)")
    p.add_argument("--cpu-seconds", type=float, default=10.0,
                   help="target CPU time of each oracle baseline sample")
    p.add_argument("--workload", choices=("rmat17", "batch256", "serving", "rmat22", "quality"),
                   default="rmat17",
                   help="rmat17: the full line (headline plus the other legs); batch256, serving, "
                        "rmat22: one leg alone, printed as its own line; quality: the theta sweep, "
                        "Exact vs GreedyReplace and BaselineGreedy vs AdvancedGreedy studies")
    p.add_argument("--requests", type=int, default=16,
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


def gpu_index(local_rank: int) -> int:
    first = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    return int(first) if first.isdigit() else local_rank


# --------------------------------------------------------------------------------------------
# roofline accounting
# --------------------------------------------------------------------------------------------

def algorithmic_bytes(stats: dict, tier: int, n_seeds: int) -> float:
    """Bytes the method must move for the samples one kernel tier finished, per sample
    8|R| (the row-offset pair of every reached vertex) + 8 E_R (target and threshold of every
    examined edge) + 8 |R \\ S| (one uint64 counter update per reached non-seed)."""
    r = stats["tier_reached"][tier]
    e = stats["tier_examined_edges"][tier]
    s = stats["tier_samples"][tier] * n_seeds
    return 8.0 * r + 8.0 * e + 8.0 * (r - s)


def algorithmic_bytes_live_targets(stats: dict, tier: int, n_seeds: int) -> float:
    """The same with a target read only for live edges (how the kernels read the graph):
    8|R| + 4 E_R + 4 L + 8 |R \\ S|."""
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


def profile_fields(kernel: str, workload: str = WORKLOAD) -> dict:
    """'key: value' header lines of the committed ncu summary profiles/<kernel>_<workload>.md."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return {}
    out = {}
    for line in open(path):
        k, sep, v = line.partition(":")
        if sep and k and k[0].islower() and all(c.islower() or c.isdigit() or c == "_" for c in k):
            out[k] = v.strip()
    return out


def ncu_traffic(kernel: str, workload: str = WORKLOAD):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken on the
    current kernel sources ('source_hash:' and 'dram_bytes_per_launch:' lines); None otherwise."""
    f = profile_fields(kernel, workload)
    if f.get("source_hash") != kernel_source_hash() or "dram_bytes_per_launch" not in f:
        return None
    return float(f["dram_bytes_per_launch"])


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def roofline_of(prof: dict, stats: dict, n_seeds: int, workload: str = WORKLOAD) -> dict:
    """Roofline of the sample kernel with the most device time: algorithmic bytes per launch
    (from the kernels' own work counters) over its average CUDA-event launch time, against the
    measured HBM copy bandwidth. `bound` names what limits the kernel: HBM when its DRAM traffic
    (ncu) is of the order of the algorithmic bytes, instruction issue when the graph is served
    from L2 (DRAM traffic far below the algorithmic bytes)."""
    kind, tier, kname = max(SAMPLE_KINDS, key=lambda k: prof[k[0]]["ms"])
    kp = prof[kind]
    launches = max(kp["launches"], 1)
    avg_ms = kp["ms"] / launches
    alg = algorithmic_bytes(stats, tier, n_seeds) / launches
    alg_live = algorithmic_bytes_live_targets(stats, tier, n_seeds) / launches
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    achieved = alg / (avg_ms * 1e-3) / 1e9
    traffic = ncu_traffic(kname, workload)
    fields = profile_fields(kname, workload)
    bound = "hbm"
    if traffic is not None and traffic < 0.25 * alg:
        bound = "issue"
    total = sum(v["ms"] for v in prof.values())
    out = {"kernel": kname, "bound": bound, "achieved": achieved, "peak": peak,
           "peak_source": src, "unit": "GB/s", "frac": achieved / peak,
           "frac_of": f"{src} HBM copy bandwidth", "traffic": traffic,
           "algorithmic_bytes_per_launch": alg,
           "algorithmic_bytes_per_launch_live_targets": alg_live,
           "frac_live_targets": alg_live / (avg_ms * 1e-3) / 1e9 / peak,
           "avg_launch_ms": avg_ms, "launches": kp["launches"],
           "share_of_device_time": kp["ms"] / max(total, 1e-9),
           "kernel_ms": {k: round(v["ms"], 3) for k, v in prof.items()}}
    if fields.get("source_hash") == kernel_source_hash():
        # the other ncu figures of the same capture (issue-slot use, L2 throughput and hit rate,
        # warp execution efficiency, L2 -> SM bytes per launch)
        out["ncu"] = {k: float(v) for k, v in fields.items()
                      if k not in ("source_hash", "dram_bytes_per_launch")}
    return out


def sum_stats(acc, st):
    if acc is None:
        return {k: (list(v) if isinstance(v, list) else v) for k, v in st.items()}
    for k, v in st.items():
        acc[k] = [a + b for a, b in zip(acc[k], v)] if isinstance(v, list) else acc[k] + v
    return acc


# --------------------------------------------------------------------------------------------
# CPU baselines and the reference arm (the oracle as it stands, on the host cores)
# --------------------------------------------------------------------------------------------

def _oracle_rate(q, threads: int, seconds: float):
    from oracle import oracle as O

    with O.threads(threads):
        probe = 100 * threads
        t = time.perf_counter()
        O.decrease(q.graph, q.seeds, [], probe, q.key, 0)
        per = (time.perf_counter() - t) / probe
        count = int(max(probe, min(q.theta, seconds / max(per, 1e-8))))
        t = time.perf_counter()
        O.decrease(q.graph, q.seeds, [], count, q.key, 0)
        dt = time.perf_counter() - t
    return count / dt, count, dt


def cpu_baseline(q, seconds: float):
    """The oracle as it stands on a bounded sample of the workload (the first `count` sampled
    graphs of round 0, sized to take about `seconds`): on all host cores (its thread-parallel
    sample loop) and on one core."""
    from oracle import oracle as O

    O.lib()
    cores = os.cpu_count() or 1
    v_all, c_all, t_all = _oracle_rate(q, cores, seconds)
    v_one, c_one, t_one = _oracle_rate(q, 1, seconds)
    return {"value": v_all, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"round 0, samples 0..{c_all - 1} of theta={q.theta} ({t_all:.1f} s, "
                      f"{cores} threads)",
            "single_core": {"value": v_one, "cores": 1,
                            "sample": f"round 0, samples 0..{c_one - 1} ({t_one:.1f} s)"}}


def run_reference(args, q, rank):
    """The oracle timed on all host cores on the same workload, metric and unit; each step is a
    bounded sample (a range of sampled graphs of one round)."""
    from oracle import oracle as O

    if rank != 0:
        return
    O.lib()
    cores = os.cpu_count() or 1
    with O.threads(cores):
        t = time.perf_counter()
        O.decrease(q.graph, q.seeds, [], 50 * cores, q.key, 0)
        per = (time.perf_counter() - t) / (50 * cores)
        per_step = int(max(100, min(q.theta, args.ref_step_seconds / max(per, 1e-8))))
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
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} sampled graphs of one round per step, "
                                       f"{cores} threads"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(q):
    return {"workload": WORKLOAD, "graph": "R-MAT scale 17, m=2^20, (0.57,0.19,0.19,0.05), WC",
            "n": q.graph.n, "m": q.graph.m, "seeds": int(len(q.seeds)), "b": q.b,
            "theta": q.theta, "samples_per_step": q.b * q.theta,
            "l2": "flushed between steps (512 MiB write outside the step events)"}


# --------------------------------------------------------------------------------------------
# legs
# --------------------------------------------------------------------------------------------

def leg_batch(steps: int, warmup: int, key_offset: int = 0) -> dict:
    """256 independent AdvancedGreedy queries (Chung-Lu, n log-uniform in [1e3, 2e5], mean degree
    U[5,20], TR probabilities, |S| U[5,100], b=20, theta=2e4): one batched call per step vs the
    same queries one imin_advanced_greedy call at a time (cutoffs tuned before timing); every
    result must be identical."""
    import numpy as np
    import torch
    from paper_2302_13529_gb300 import imin, workloads as W

    t0 = time.perf_counter()
    qs = W.batch_queries(256)
    gen_s = time.perf_counter() - t0
    hs = [imin.load_graph(q.graph) for q in qs]
    items = [(h, q.seeds, q.b, q.theta, q.key + key_offset) for h, q in zip(hs, qs)]
    samples = sum(q.b * q.theta for q in qs)  # every query runs b rounds (n - |S| >= b here)
    chunk = imin.autotune_batch(items, 0)  # queue granularity, tuned outside the timing
    for _ in range(max(warmup, 1)):
        imin.batch_advanced_greedy(items)
    torch.cuda.synchronize()
    launches0 = imin.launch_count()
    times = []
    res = None
    for _ in range(steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = imin.batch_advanced_greedy(items)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    launches = imin.launch_count() - launches0
    st = imin.last_stats()
    imin.profile_read(reset=True)
    imin.profile_enable(True)
    imin.batch_advanced_greedy(items)
    imin.profile_enable(False)
    prof = imin.profile_read(reset=True)
    for h, it in zip(hs, items):  # the plain calls' per-graph cutoff tuning stays out of their timing
        imin.autotune(h, it[1], it[4])
    imin.advanced_greedy(*items[0])
    torch.cuda.synchronize()
    t = time.perf_counter()
    plain = [imin.advanced_greedy(*it) for it in items]
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t
    same = all(np.array_equal(a, b) for a, b in zip(res, plain))
    batched_s = min(times)
    for h in hs:
        h.close()
    return {"workload": "batch256-chunglu-tr-advanced-greedy", "queries": len(qs), "b": 20,
            "theta": 20000, "samples_per_call": samples,
            "total_edges": int(sum(q.graph.m for q in qs)), "generation_s": round(gen_s, 1),
            "batched": {"value": samples / batched_s, "unit": "samples/s", "seconds": batched_s,
                        "calls": steps, "gpu_launches_per_call": launches / max(steps, 1),
                        "samples_per_work_item": chunk},
            "one_query_per_launch": {"value": samples / plain_s, "unit": "samples/s",
                                     "seconds": plain_s, "cutoff": "autotuned per graph before timing"},
            "batched_over_plain": plain_s / batched_s, "bit_exact_vs_plain": same,
            "kernel_ms": {k: round(v["ms"], 3) for k, v in prof.items()},
            "work": {"reached_per_sample": st["reached"] / max(st["samples"], 1),
                     "examined_edges_per_sample": st["examined_edges"] / max(st["samples"], 1)}}


def leg_rmat22(b=None, theta=None, key_offset: int = 0) -> dict:
    """The large single query: R-MAT n=2^22, m=2^26, WC, |S|=200, b=200, theta=2*10^5, rounds
    captured in one CUDA graph, inputs resident on the device. Warm-up: one 2-round query (module
    load, cutoff tuning, allocator pools); then one AdvancedGreedy and one GreedyReplace query,
    each timed with CUDA events on the launching stream."""
    import torch
    from paper_2302_13529_gb300 import imin, workloads as W

    t0 = time.perf_counter()
    q = W.rmat22_query()
    if b is not None or theta is not None:
        q = W.Query(q.graph, q.seeds, b if b is not None else q.b, theta if theta is not None else q.theta,
                    q.key)
    gen_s = time.perf_counter() - t0
    key = q.key + key_offset
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
    gh.close()
    return {"workload": "rmat22-wc", "n": q.graph.n, "m": q.graph.m, "seeds": len(q.seeds),
            "b": q.b, "theta": q.theta, "warp_block_cutoff": cutoff,
            "generation_s": round(gen_s, 1), "l2": "graph (528 MB) larger than L2",
            "ag_wall_s": walls["ag"], "gr_wall_s": walls["gr"],
            "ag_samples_per_s": samples / walls["ag"], "ag_samples": samples,
            "gr_samples": walls["gr_stats"]["samples"],
            "work": {"reached_per_sample": st["reached"] / max(samples, 1),
                     "examined_edges_per_sample": st["examined_edges"] / max(samples, 1),
                     "tier_samples": st["tier_samples"]}}


def leg_serving(requests: int, seed: int = 5000, max_class_samples: int = 0) -> dict:
    """Requests against the R-MAT 2^17 (m=2^20) and R-MAT 2^22 (m=2^26) WC graphs held resident:
    each picks a graph with probability 1/2, |S| ~ U[10, 500], b ~ U[10, 100],
    theta ~ U[1e4, 1e5] (AdvancedGreedy).
      serial   every request run alone, one after another (imin_advanced_greedy): its service
               time and the saturated serial throughput;
      burst    all requests submitted at once to the continuous-batching server: its saturated
               throughput;
      poisson  the same requests with Poisson arrivals at 80 % of the serial saturation rate,
               through the server (latency p50/p99), and through a one-at-a-time FIFO queue
               whose latencies follow from the same arrival times and the measured service
               times (finish_i = max(arrival_i, finish_{i-1}) + service_i)."""
    import threading

    import numpy as np
    import torch
    from paper_2302_13529_gb300 import imin, workloads as W

    graphs = [W.rmat17_query().graph, W.rmat22_query().graph]
    hs = [imin.load_graph(g) for g in graphs]
    reqs = W.serving_requests(requests, seed)
    samples = sum(r.b * r.theta for r in reqs)

    def serve(arrivals):
        lat = [None] * len(reqs)
        with imin.Server(max_class_samples=max_class_samples) as srv:
            t0 = time.perf_counter()
            tickets = [None] * len(reqs)

            def submitter():
                for i, r in enumerate(reqs):
                    wait = arrivals[i] - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(wait)
                    tickets[i] = srv.submit(0, hs[r.gi], r.seeds, r.b, r.theta, r.key)

            th = threading.Thread(target=submitter)
            th.start()
            th.join()
            for i, r in enumerate(reqs):
                _, lat[i] = srv.wait(tickets[i], capacity=r.b)
            elapsed = time.perf_counter() - t0
            st = srv.stats()
        return elapsed, np.array(lat), st

    for r in reqs:  # every graph / seed-set size class tuned before anything is timed
        imin.advanced_greedy(hs[r.gi], r.seeds, 1, 1000, r.key)
    torch.cuda.synchronize()
    service = []
    for r in reqs:
        t = time.perf_counter()
        imin.advanced_greedy(hs[r.gi], r.seeds, r.b, r.theta, r.key)
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t)
    serial_s = sum(service)
    burst_s, burst_lat, _ = serve([0.0] * len(reqs))
    rate = 0.8 * len(reqs) / serial_s  # requests per second at 80 % of serial saturation
    gaps = np.random.default_rng(seed + 1000).exponential(1.0 / rate, size=len(reqs))
    arrivals = np.cumsum(gaps) - gaps[0]
    poisson_s, lat, st = serve(list(arrivals))
    fifo, finish = [], 0.0
    for a, sv in zip(arrivals, service):
        finish = max(a, finish) + sv
        fifo.append(1e3 * (finish - a))
    fifo = np.array(fifo)
    for h in hs:
        h.close()
    pct = lambda a, p: float(np.percentile(a, p))
    return {"workload": "serving-rmat17-rmat22-advanced-greedy", "requests": len(reqs),
            "full_configuration_requests": 2000, "samples": samples,
            "value": samples / poisson_s, "unit": "samples/s", "seconds": poisson_s,
            "arrivals": f"Poisson at 80% of the serial saturation rate ({rate:.3f} req/s)",
            "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": float(lat.max())},
            "fifo_serial_latency_ms": {"p50": pct(fifo, 50), "p99": pct(fifo, 99), "max": float(fifo.max())},
            "burst": {"seconds": burst_s, "samples_per_s": samples / burst_s,
                      "p50_ms": pct(burst_lat, 50), "p99_ms": pct(burst_lat, 99)},
            "serial_one_query_at_a_time": {"value": samples / serial_s, "unit": "samples/s",
                                           "seconds": serial_s, "requests": len(reqs)},
            "burst_over_serial": serial_s / burst_s,
            "p99_serial_over_server": pct(fifo, 99) / pct(lat, 99),
            "server": st}


def leg_theta_sweep(eval_theta: int = 100_000) -> dict:
    """The paper's theta sensitivity study (Sec. 5, "Varying the Number of Sampled Graphs": TR
    model, b = 20, 10 random seeds, theta in {10^3, 10^4, 10^5}, GreedyReplace's expected spread
    and running time) on two synthetic stand-ins: R-MAT 2^17 / 2^20 and Chung-Lu n = 10^5,
    m = 10^6, both with TR probabilities. Each blocker set's spread is simulated with
    `eval_theta` samples on an independent key; the decrease ratio is spread(theta_prev) /
    spread(theta) - 1."""
    import numpy as np
    import torch
    from paper_2302_13529_gb300 import imin, workloads as W

    rp, col = W.rmat(17, 1 << 20, W.RMAT_ABCD, 1102)
    g1 = W.Graph(1 << 17, rp, col, W.tr_thresholds(len(col), 1103), "rmat17-tr")
    rp, col = W.chung_lu(100_000, 1_000_000, 2.1, 1104)
    g2 = W.Graph(100_000, rp, col, W.tr_thresholds(len(col), 1105), "chunglu-1e5-tr")
    out = {"model": "TR", "b": 20, "seeds": 10, "eval_theta": eval_theta, "graphs": {}}
    for g in (g1, g2):
        gh = imin.load_graph(g)
        seeds = W.uniform_seeds(g.n, 10, 1106)
        key = W.query_key(1107)
        ev_key = W.query_key(1108)
        rows, prev = [], None
        imin.greedy_replace(gh, seeds, 20, 1000, key)  # warm-up and cutoff tuning
        for theta in (1000, 10_000, 100_000):
            torch.cuda.synchronize()
            t = time.perf_counter()
            B = imin.greedy_replace(gh, seeds, 20, theta, key)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t
            sp = imin.estimate_spread(gh, seeds, B, eval_theta, ev_key) / eval_theta
            rows.append({"theta": theta, "gr_seconds": secs, "expected_spread": sp,
                         "decrease_ratio_vs_previous": (prev / sp - 1.0) if prev else None})
            prev = sp
        out["graphs"][g.name] = {"n": g.n, "m": g.m, "runs": rows,
                                 "no_blockers_spread": imin.estimate_spread(gh, seeds, [], eval_theta, ev_key)
                                 / eval_theta}
        gh.close()
    return out


def leg_exact_small(bmax: int = 3, r: int = 10_000) -> dict:
    """Exact vs GreedyReplace on small graphs (the paper's Tables 5-6 compare them on 100-vertex
    extracts of EmailCore with 10 random seeds and theta = r = 10^4, TR and WC): a directed
    Chung-Lu graph with n = 100, m = 800 under TR and WC, 10 seeds, b = 1..bmax; the spread of
    each result simulated with 10^5 samples on an independent key, and both running times."""
    import torch
    from paper_2302_13529_gb300 import imin, workloads as W

    rp, col = W.chung_lu(100, 800, 2.1, 1201)
    graphs = {"TR": W.Graph(100, rp, col, W.tr_thresholds(len(col), 1202)),
              "WC": W.Graph(100, rp, col, W.wc_thresholds(col, 100))}
    seeds = W.uniform_seeds(100, 10, 1203)
    key, ev_key = W.query_key(1204), W.query_key(1205)
    out = {"n": 100, "m": 800, "seeds": 10, "r": r, "theta": r, "models": {}}
    for name, g in graphs.items():
        gh = imin.load_graph(g)
        imin.greedy_replace(gh, seeds, 1, 1000, key)
        rows = []
        for b in range(1, bmax + 1):
            torch.cuda.synchronize()
            t = time.perf_counter()
            E = imin.exact_blockers(gh, seeds, b, r, key)
            torch.cuda.synchronize()
            t_exact = time.perf_counter() - t
            t = time.perf_counter()
            G = imin.greedy_replace(gh, seeds, b, r, key)
            torch.cuda.synchronize()
            t_gr = time.perf_counter() - t
            se = imin.estimate_spread(gh, seeds, E, 100_000, ev_key) / 1e5
            sg = imin.estimate_spread(gh, seeds, G, 100_000, ev_key) / 1e5
            rows.append({"b": b, "exact_seconds": t_exact, "gr_seconds": t_gr, "exact_spread": se,
                         "gr_spread": sg, "gr_over_exact_spread": sg / se,
                         "exact": [int(x) for x in E], "gr": [int(x) for x in G]})
        out["models"][name] = rows
        gh.close()
    return out


def leg_baseline_greedy(b: int = 10, r: int = 10_000) -> dict:
    """AdvancedGreedy and GreedyReplace against BaselineGreedy (Alg. 1, every candidate scored by
    r simulations per round) on the small Chung-Lu workload (n = 2,000, m = 10^4, WC, |S| = 10),
    b rounds, theta = r; the paper reports AG and GR >= 3 orders of magnitude faster at b = 10.
    BaselineGreedy must return AdvancedGreedy's list (the same samples, Cor. 1)."""
    import torch
    from paper_2302_13529_gb300 import imin, workloads as W

    q = W.tiny_chung_lu_query()
    gh = imin.load_graph(q.graph)
    imin.advanced_greedy(gh, q.seeds, 1, 1000, q.key)
    times, res = {}, {}
    for name, fn in (("baseline_greedy", imin.baseline_greedy), ("advanced_greedy", imin.advanced_greedy),
                     ("greedy_replace", imin.greedy_replace)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        res[name] = [int(x) for x in fn(gh, q.seeds, b, r, q.key)]
        torch.cuda.synchronize()
        times[name] = time.perf_counter() - t
    gh.close()
    return {"graph": "chunglu n=2000 m=10000 WC", "seeds": 10, "b": b, "r": r, "seconds": times,
            "speedup_ag_over_bg": times["baseline_greedy"] / times["advanced_greedy"],
            "speedup_gr_over_bg": times["baseline_greedy"] / times["greedy_replace"],
            "bg_equals_ag": res["baseline_greedy"] == res["advanced_greedy"]}


def leg_line(name: str, leg: dict, world: int) -> dict:
    """A leg run alone (--workload batch256 / rmat22 / serving / quality), as its own bench line."""
    if name == "quality":
        bg = leg["baseline_greedy"]
        return {"metric": METRIC, "value": 1.0 / bg["seconds"]["advanced_greedy"], "unit": "queries/s",
                "n_gpus": world, "steps": 1, "warmup": 1,
                "ms_per_step": 1e3 * bg["seconds"]["advanced_greedy"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "uint32", "data": "synthetic",
                "config": {"workload": "quality-studies"}, name: leg}
    if name == "batch256":
        v, ms = leg["batched"]["value"], 1e3 * leg["batched"]["seconds"]
    elif name == "rmat22":
        v, ms = leg["ag_samples_per_s"], 1e3 * leg["ag_wall_s"]
    else:
        v, ms = leg["value"], 1e3 * leg["seconds"]
    return {"metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": world, "steps": 1,
            "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "uint32", "data": "synthetic",
            "config": {"workload": leg["workload"]}, name: leg}


# --------------------------------------------------------------------------------------------
# main
# --------------------------------------------------------------------------------------------

def main(argv=None):
    args = parse_args(argv)
    rank, world, local_rank = dist_env()
    from paper_2302_13529_gb300 import workloads as W

    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        if args.impl == "ours" and torch.cuda.is_available():
            torch.cuda.set_device(local_rank)
            tdist.init_process_group("nccl")
        else:
            tdist.init_process_group("gloo")
        dist = tdist

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
    if args.workload != "rmat17":
        leg = {"batch256": lambda: leg_batch(max(args.steps, 1), args.warmup, rank),
               "rmat22": lambda: leg_rmat22(args.b, args.theta, rank),
               "serving": lambda: leg_serving(args.requests, 5000 + rank),
               "quality": lambda: {"theta_sweep": leg_theta_sweep(), "exact_small": leg_exact_small(),
                                   "baseline_greedy": leg_baseline_greedy()}}[args.workload]()
        if rank == 0:
            print(json.dumps(leg_line(args.workload, leg, world)), flush=True)
        return

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

    # timed steps: the production path (all rounds of a query in one captured CUDA graph), with
    # no profiling events in it
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stats_sum = None
    launches0 = imin.launch_count()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_index(local_rank)) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            step()
            stops[k].record(stream)
            stats_sum = sum_stats(stats_sum, imin.last_stats())
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = imin.launch_count() - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, stops)]
    local_s = sum(step_ms) / 1e3
    samples_local = q.b * q.theta * args.steps
    value, slowest = aggregate(local_s, samples_local, world, reduce_max, reduce_sum)
    ms_per_step = 1e3 * slowest / args.steps

    # per-kernel times: the same K steps once more, untimed, with an event-record node on each
    # side of every kernel inside the captured graphs (the nodes add about 1 % to a step)
    imin.profile_read(reset=True)
    imin.profile_enable(True)
    prof_stats = None
    for k in range(args.steps):
        flush.fill_(float(k))
        step()
        prof_stats = sum_stats(prof_stats, imin.last_stats())
    torch.cuda.synchronize()
    imin.profile_enable(False)
    prof = imin.profile_read(reset=True)
    roofline = roofline_of(prof, prof_stats, len(q.seeds))
    if sum(v["ms"] for v in prof.values()) <= 0:
        # event nodes inside graphs gave no times: time one query with the graphs off instead
        os.environ["IMIN_NO_GRAPHS"] = "1"
        imin.profile_enable(True)
        step()
        torch.cuda.synchronize()
        imin.profile_enable(False)
        del os.environ["IMIN_NO_GRAPHS"]
        prof = imin.profile_read(reset=True)
        roofline = roofline_of(prof, imin.last_stats(), len(q.seeds))
        roofline["timing"] = "separate untimed query without CUDA graphs"
    else:
        roofline["timing"] = ("CUDA events inside the graphs of a separate untimed pass of the same "
                              "steps, right after the timed ones")

    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "uint32",
            "data": "synthetic", "config": dict(config_of(q), warp_block_cutoff=cutoff),
            "roofline": roofline, "gpu_launches": launches,
            "work": {"reached_per_sample": stats_sum["reached"] / stats_sum["samples"],
                     "examined_edges_per_sample": stats_sum["examined_edges"] / stats_sum["samples"],
                     "live_edges_per_sample": stats_sum["live_edges"] / stats_sum["samples"],
                     "live_edges_per_s": value * stats_sum["live_edges"] / stats_sum["samples"],
                     "examined_edges_per_s": value * stats_sum["examined_edges"] / stats_sum["samples"],
                     "tier_samples": stats_sum["tier_samples"]},
            "ag_wall_s": ms_per_step / 1e3}
    clocks = clk.summary()
    if clocks is not None:
        line["clocks"] = clocks

    # GreedyReplace wall time (one query, device-resident inputs, CUDA events)
    ag_blockers = out_d.cpu().numpy().copy()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    imin.greedy_replace(gh, seeds_d, q.b, q.theta, key, out=out_d)
    e1.record(stream)
    torch.cuda.synchronize()
    line["gr_wall_s"] = e0.elapsed_time(e1) / 1e3
    line["gr_samples"] = imin.last_stats()["samples"]
    gr_blockers = out_d[:q.b].cpu().numpy().copy()

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
                       "includes": "graph upload + validation (a new handle each step; its "
                                   "warp/block cutoff comes from the process-wide tuning cache), "
                                   "seed upload, 50 rounds in one CUDA graph, blocker read-back"}
    gh.close()
    del flush

    if world == 1 and not args.no_extras:
        line["batched_vs_plain"] = leg_batch(2, 1)
        line["large_query"] = leg_rmat22()
        line["serving"] = leg_serving(args.requests)
        line["quality"] = {"theta_sweep": leg_theta_sweep(), "exact_small": leg_exact_small(),
                           "baseline_greedy": leg_baseline_greedy()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(q, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
