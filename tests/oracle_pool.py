"""Run the CPU oracle over sample ranges in a spawned process pool (full-size parity checks).

The oracle is single-threaded; Alg. 2's counters are integer sums over samples, so splitting
[0, theta) into ranges and adding the partial counters gives exactly the same result.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_G = None


def _init(n, row_ptr, col, thr):
    global _G
    from paper_2302_13529_gb300.workloads import Graph
    _G = Graph(n, row_ptr, col, thr)


def _work(args):
    from oracle import oracle as O
    seeds, blocked, j0, cnt, key, round_ = args
    return O.decrease(_G, seeds, blocked, cnt, key, round_, j0)


def workers() -> int:
    return max(1, min(32, (os.cpu_count() or 2)))


def decrease(g, seeds, blocked, theta, key, round_, nproc=None, chunks_per_proc=4):
    """Alg. 2 counters over samples [0, theta), computed by the oracle in parallel."""
    nproc = nproc or workers()
    nchunk = max(1, min(theta, nproc * chunks_per_proc))
    bounds = np.linspace(0, theta, nchunk + 1).astype(np.int64)
    tasks = [(np.asarray(seeds, np.int32), np.asarray(blocked if blocked is not None else [], np.int32),
              int(bounds[i]), int(bounds[i + 1] - bounds[i]), int(key), int(round_))
             for i in range(nchunk) if bounds[i + 1] > bounds[i]]
    ctx = mp.get_context("spawn")
    with ctx.Pool(nproc, initializer=_init, initargs=(g.n, g.row_ptr, g.col, g.thr)) as pool:
        parts = pool.map(_work, tasks)
    return np.sum(parts, axis=0, dtype=np.uint64)
