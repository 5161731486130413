"""GPU parity of the simulated expected spread (Def. 3): the CUDA library's sum of |R| over the
sampled graphs must equal the oracle's exactly (integer counts on the same Philox stream)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2302_13529_gb300 import workloads as W
from tests.test_gpu_parity import _small_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("i", range(12))
def test_spread_small_graphs(cuda_lib, i):
    g, seeds, blocked = _small_case(i)
    gh = cuda_lib.load_graph(g)
    for theta, key, rnd in ((1, 3, 0), (53, 99, 2), (3000, 0xC0FFEE, 9)):
        assert cuda_lib.estimate_spread(gh, seeds, blocked, theta, key, rnd) == \
            O.spread(g, seeds, blocked, theta, key, rnd), (i, theta)


def test_spread_chung_lu_and_blockers(cuda_lib):
    q = W.tiny_chung_lu_query()
    gh = cuda_lib.load_graph(q.graph)
    B = O.advanced_greedy(q.graph, q.seeds, 5, 2000, q.key)
    for blocked in ([], list(B)):
        got = cuda_lib.estimate_spread(gh, q.seeds, blocked, 10_000, 77, 0)
        assert got == O.spread(q.graph, q.seeds, blocked, 10_000, 77, 0)
    # blocking the estimator's choices lowers the spread (statistically, by a wide margin here)
    assert cuda_lib.estimate_spread(gh, q.seeds, list(B), 10_000, 78) < \
        cuda_lib.estimate_spread(gh, q.seeds, [], 10_000, 78)


def test_spread_full_size_rmat17(cuda_lib):
    q = W.rmat17_query()
    gh = cuda_lib.load_graph(q.graph)
    got = cuda_lib.estimate_spread(gh, q.seeds, [], 10_000, q.key, 1)
    assert got == O.spread(q.graph, q.seeds, [], 10_000, q.key, 1)
    st = cuda_lib.last_stats()
    assert st["samples"] == 10_000 and st["reached"] == got


def test_spread_large_graph_global_bitmap(cuda_lib):
    g = W.graph_rmat_wc(19, 1 << 20, seed=91)
    seeds = W.uniform_seeds(g.n, 30, 92)
    gh = cuda_lib.load_graph(g)
    assert cuda_lib.estimate_spread(gh, seeds, [3, 4], 2000, 93, 1) == O.spread(g, seeds, [3, 4], 2000, 93, 1)


def test_spread_invalid_arguments(cuda_lib):
    q = W.tiny_chung_lu_query()
    gh = cuda_lib.load_graph(q.graph)
    with pytest.raises(cuda_lib.IminError):
        cuda_lib.estimate_spread(gh, q.seeds, [int(q.seeds[0])], 10, 1)  # blocked seed
    with pytest.raises(cuda_lib.IminError):
        cuda_lib.estimate_spread(gh, q.seeds, [], 0, 1)  # theta = 0
    with pytest.raises(cuda_lib.IminError):
        cuda_lib.estimate_spread(gh, [q.graph.n], [], 10, 1)  # seed out of range
    # all non-seeds blocked: only the seeds are ever active
    rest = [v for v in range(q.graph.n) if v not in set(q.seeds.tolist())]
    assert cuda_lib.estimate_spread(gh, q.seeds, rest, 100, 1) == 100 * len(q.seeds)
