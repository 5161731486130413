"""The comparison algorithms of Sec. 5 on the GPU (through the C ABI) against the oracle:
simulated spread of many blocker sets, BaselineGreedy (Alg. 1), Exact, OutDegree and Rand."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2302_13529_gb300 import workloads as W
from tests.test_oracle_baselines import _small
from tests.test_oracle_pins import TOY

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(4))
def test_spread_sets_small_graphs(cuda_lib, seed):
    g, seeds = _small(seed)
    rng = np.random.default_rng(seed)
    rest = [v for v in range(g.n) if v not in seeds]
    base = [int(rng.choice(rest))]
    others = [v for v in rest if v not in base]
    sets = [[int(x) for x in rng.choice(others, 2, replace=False)] for _ in range(7)]
    gh = cuda_lib.load_graph(g)
    got = cuda_lib.estimate_spread_sets(gh, seeds, base, sets, 999, 5 + seed, 3)
    assert np.array_equal(got, O.spread_sets(g, seeds, base, sets, 999, 5 + seed, 3))


def test_spread_sets_chung_lu_and_lt(cuda_lib):
    q = W.tiny_chung_lu_query()
    rest = np.setdiff1d(np.arange(q.graph.n), q.seeds)
    sets = [[int(v)] for v in rest[:40]] + [[]] * 0
    gh = cuda_lib.load_graph(q.graph)
    got = cuda_lib.estimate_spread_sets(gh, q.seeds, [], sets, 2000, q.key, 1)
    assert np.array_equal(got, O.spread_sets(q.graph, q.seeds, [], sets, 2000, q.key, 1))
    g_lt = W.Graph(q.graph.n, q.graph.row_ptr, q.graph.col, W.lt_wc_weights(q.graph.col, q.graph.n))
    hl = cuda_lib.load_graph(g_lt, model="lt")
    got = cuda_lib.estimate_spread_sets(hl, q.seeds, [], sets, 2000, q.key, 1)
    assert np.array_equal(got, O.spread_sets(g_lt, q.seeds, [], sets, 2000, q.key, 1, model="lt"))
    # set_size 0: one set that blocks nothing is the plain spread
    assert cuda_lib.estimate_spread_sets(gh, q.seeds, [], np.zeros((1, 0), np.int32), 2000, q.key, 1)[0] == \
        cuda_lib.estimate_spread(gh, q.seeds, [], 2000, q.key, 1)


def test_baseline_greedy_against_oracle_and_advanced_greedy(cuda_lib):
    """BaselineGreedy on the GPU equals the oracle's, and -- blocking u removes exactly what u
    dominates in each sample (Cor. 1) -- equals AdvancedGreedy with theta = r."""
    gh = cuda_lib.load_graph(TOY)
    assert [int(x) for x in cuda_lib.baseline_greedy(gh, [0], 2, 20_000, 3)] == [4, 1]
    for seed in range(3):
        g, seeds = _small(seed)
        gh = cuda_lib.load_graph(g)
        got = [int(x) for x in cuda_lib.baseline_greedy(gh, seeds, 3, 500, 40 + seed)]
        assert got == [int(x) for x in O.baseline_greedy(g, seeds, 3, 500, 40 + seed)]
        assert got == [int(x) for x in cuda_lib.advanced_greedy(gh, seeds, 3, 500, 40 + seed)]
    q = W.tiny_chung_lu_query()
    gh = cuda_lib.load_graph(q.graph)
    bg = [int(x) for x in cuda_lib.baseline_greedy(gh, q.seeds, 2, 1000, q.key)]
    assert bg == [int(x) for x in cuda_lib.advanced_greedy(gh, q.seeds, 2, 1000, q.key)]


def test_exact_against_oracle(cuda_lib):
    gh = cuda_lib.load_graph(TOY)
    assert [int(x) for x in cuda_lib.exact_blockers(gh, [0], 1, 5000, 8)] == [4]
    assert [int(x) for x in cuda_lib.exact_blockers(gh, [0], 2, 5000, 8)] == [1, 3]
    for seed in range(3):
        g, seeds = _small(seed, n=14)
        gh = cuda_lib.load_graph(g)
        for b in (1, 2, 3):
            got = [int(x) for x in cuda_lib.exact_blockers(gh, seeds, b, 300, seed)]
            assert got == [int(x) for x in O.exact(g, seeds, b, 300, seed)], (seed, b)


def test_out_degree_and_random(cuda_lib):
    q = W.tiny_chung_lu_query()
    gh = cuda_lib.load_graph(q.graph)
    for b in (0, 1, 10, 3000):
        assert np.array_equal(cuda_lib.out_degree_blockers(gh, q.seeds, b), O.out_degree_blockers(q.graph, q.seeds, b))
        for key in (1, 99):
            assert np.array_equal(cuda_lib.random_blockers(gh, q.seeds, b, key),
                                  O.random_blockers(q.graph.n, q.seeds, b, key))


def test_sets_are_validated(cuda_lib):
    from paper_2302_13529_gb300.imin import IminError
    gh = cuda_lib.load_graph(TOY)
    for sets in ([[0]], [[1, 1]], [[9]], [[2]]):  # a seed, a repeat, out of range, a blocked vertex
        with pytest.raises(IminError) as e:
            cuda_lib.estimate_spread_sets(gh, [0], [2], sets, 10, 1)
        assert e.value.code == -1


def test_comparison_algorithms_reject_bad_arguments_and_take_device_buffers(cuda_lib):
    import torch
    from paper_2302_13529_gb300.imin import IminError
    q = W.tiny_chung_lu_query()
    gh = cuda_lib.load_graph(q.graph)
    for f in (cuda_lib.baseline_greedy, cuda_lib.exact_blockers):
        with pytest.raises(IminError):
            f(gh, q.seeds, -1, 10, 1)
        with pytest.raises(IminError):
            f(gh, q.seeds, 1, 0, 1)  # r = 0
        assert len(f(gh, q.seeds, 0, 10, 1)) == 0
    with pytest.raises(IminError):
        cuda_lib.exact_blockers(gh, q.seeds, 6, 10, 1)  # C(1990, 6) sets: beyond the limit
    # device seeds, sets and output
    rest = np.setdiff1d(np.arange(q.graph.n), q.seeds)[:16].astype(np.int32)
    sets_d = torch.from_numpy(rest.reshape(8, 2)).cuda()
    out_d = torch.zeros(8, dtype=torch.uint64, device="cuda")
    seeds_d = torch.from_numpy(q.seeds).cuda()
    s_ptr = cuda_lib._ptr(sets_d, np.int32)[0]
    o_ptr = cuda_lib._ptr(out_d, np.uint64)[0]
    sd_ptr = cuda_lib._ptr(seeds_d, np.int32)[0]
    rc = cuda_lib.lib().imin_estimate_spread_sets(gh.handle, sd_ptr, len(q.seeds), None, 0, s_ptr, 8, 2, 500,
                                                  q.key, 2, o_ptr, cuda_lib._stream(None))
    assert rc == 0
    assert np.array_equal(out_d.cpu().numpy(), O.spread_sets(q.graph, q.seeds, [], rest.reshape(8, 2), 500, q.key, 2))
