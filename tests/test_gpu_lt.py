"""The linear-threshold model (Sec. 4.5, the standard triggering model) on the GPU, through the C
ABI (imin_load_graph_lt), against the oracle's LT mode, bit for bit.

Only the live-edge decision changes: edge (u, v) stays in a sample iff v's Philox word lies in
the edge's share of [0, 2^32). BFS, dominators, subtree sizes, counters, the greedy drivers,
batches, serving and the spread estimate are the IC path's, so every entry point is exercised on
LT graphs here.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2302_13529_gb300 import workloads as W
from tests import oracle_pool
from tests.test_oracle_lt import _lt_graph

pytestmark = pytest.mark.gpu


def _lt_wc(g):
    """The same graph with LT weighted-cascade shares b(u, v) = 1 / d_in(v)."""
    return W.Graph(g.n, g.row_ptr, g.col, W.lt_wc_weights(g.col, g.n), g.name + "-lt")


@pytest.mark.parametrize("i", range(10))
def test_lt_decrease_small_graphs(cuda_lib, i):
    rng = np.random.default_rng(7000 + i)
    n = int(rng.integers(6, 60))
    g = _lt_graph(n, int(rng.integers(n, 4 * n)), seed=7100 + i, certain_frac=0.3)
    seeds = [int(x) for x in rng.choice(n, int(rng.integers(1, 4)), replace=False)]
    rest = [v for v in range(n) if v not in seeds]
    blocked = [int(x) for x in rng.choice(rest, min(2, len(rest)), replace=False)]
    gh = cuda_lib.load_graph(g, model="lt")
    for theta, key, rnd in ((1, 3, 0), (333, 77, 2), (3000, 0xFEEDFACE, 9)):
        want = O.decrease(g, seeds, blocked, theta, key, rnd, model="lt")
        got = cuda_lib.estimate_decrease(gh, seeds, blocked, theta, key, rnd)
        assert np.array_equal(got, want), (i, theta)


def test_lt_chung_lu_all_entry_points(cuda_lib):
    """The small Chung-Lu workload with LT-WC shares: Alg. 2 with and without blockers,
    AdvancedGreedy, GreedyReplace, the spread estimate, and the warp/block cutoffs 0 and 400."""
    q = W.tiny_chung_lu_query()
    g = _lt_wc(q.graph)
    gh = cuda_lib.load_graph(g, model="lt")
    blocked = [int(x) for x in np.setdiff1d(np.arange(40), q.seeds)[:5]]
    for rnd, bl in ((0, []), (3, blocked)):
        want = O.decrease(g, q.seeds, bl, q.theta, q.key, rnd, model="lt")
        assert np.array_equal(cuda_lib.estimate_decrease(gh, q.seeds, bl, q.theta, q.key, rnd), want)
    ag = cuda_lib.advanced_greedy(gh, q.seeds, q.b, 4000, q.key)
    assert [int(x) for x in ag] == [int(x) for x in O.advanced_greedy(g, q.seeds, q.b, 4000, q.key, model="lt")]
    gr = cuda_lib.greedy_replace(gh, q.seeds, q.b, 4000, q.key)
    assert [int(x) for x in gr] == [int(x) for x in O.greedy_replace(g, q.seeds, q.b, 4000, q.key, model="lt")]
    assert cuda_lib.estimate_spread(gh, q.seeds, blocked, 5000, 11, 1) == \
        O.spread(g, q.seeds, blocked, 5000, 11, 1, model="lt")


@pytest.mark.parametrize("cutoff", ["0", "48", "400"])
def test_lt_cutoffs_and_fallback_tiers(cuda_lib, monkeypatch, cutoff):
    g = _lt_wc(W.graph_rmat_wc(12, 40000, seed=15))
    seeds = W.uniform_seeds(g.n, 20, seed=16)
    monkeypatch.setenv("IMIN_TIER0_VERTICES", cutoff)
    if cutoff == "48":
        monkeypatch.setenv("IMIN_CTA_EDGE_CAP", "2")  # also push samples to the whole-graph tier
    gh = cuda_lib.load_graph(g, model="lt")
    got = cuda_lib.estimate_decrease(gh, seeds, [5, 7], 3000, 77, 4)
    assert np.array_equal(got, O.decrease(g, seeds, [5, 7], 3000, 77, 4, model="lt"))


def test_lt_rmat17_full_round(cuda_lib):
    """The mid-scale R-MAT 2^17 graph with LT-WC shares, |S| = 50: one full Alg. 2 call
    (theta = 10^5) against the oracle, every counter."""
    q = W.rmat17_query()
    g = _lt_wc(q.graph)
    gh = cuda_lib.load_graph(g, model="lt")
    got = cuda_lib.estimate_decrease(gh, q.seeds, [], q.theta, q.key, 0)
    want = oracle_pool.decrease(g, q.seeds, [], q.theta, q.key, 0, model="lt")
    assert np.array_equal(got, want)


def test_lt_batch_and_server_equal_single_queries(cuda_lib):
    """LT and IC graphs mixed in one batch and in one server: each result equals the query run
    alone (and, for two of them, the oracle's)."""
    q = W.tiny_chung_lu_query()
    g_lt = _lt_wc(q.graph)
    rp, col = W.chung_lu(3000, 20000, 2.1, seed=24)
    g2 = W.Graph(3000, rp, col, W.lt_wc_weights(col, 3000))
    h_lt, h_ic, h2 = (cuda_lib.load_graph(g_lt, model="lt"), cuda_lib.load_graph(q.graph),
                      cuda_lib.load_graph(g2, model="lt"))
    items = [(h_lt, q.seeds, 4, 2000, 5), (h_ic, q.seeds, 4, 2000, 5), (h2, W.uniform_seeds(3000, 30, 1), 3, 1500, 6)]
    for batch, single in ((cuda_lib.batch_advanced_greedy, cuda_lib.advanced_greedy),
                          (cuda_lib.batch_greedy_replace, cuda_lib.greedy_replace)):
        res = batch(items)
        for it, r in zip(items, res):
            assert np.array_equal(r, single(*it))
    assert [int(x) for x in cuda_lib.batch_advanced_greedy(items)[0]] == \
        [int(x) for x in O.advanced_greedy(g_lt, q.seeds, 4, 2000, 5, model="lt")]
    with cuda_lib.Server(max_active=4) as srv:
        t = [srv.submit(0, it[0], it[1], it[2], it[3], it[4]) for it in items]
        got = [srv.wait(tk, capacity=it[2])[0] for tk, it in zip(t, items)]
    for it, r in zip(items, got):
        assert np.array_equal(r, cuda_lib.advanced_greedy(*it))


def test_lt_shares_above_one_are_rejected(cuda_lib):
    from paper_2302_13529_gb300.imin import IminError
    g = W.graph_from_edges(3, [(0, 2, 1), (1, 2, W.Fraction(1, 2))])
    with pytest.raises(IminError) as e:
        cuda_lib.load_graph(g, model="lt")  # shares 1 + 1/2 into vertex 2
    assert e.value.code == -1
    ok = W.graph_from_edges(3, [(0, 2, W.Fraction(1, 2)), (1, 2, W.Fraction(1, 2))])
    gh = cuda_lib.load_graph(ok, model="lt")
    d = cuda_lib.estimate_decrease(gh, [0], [], 1000, 3)
    assert np.array_equal(d, O.decrease(ok, [0], [], 1000, 3, model="lt"))
