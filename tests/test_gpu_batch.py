"""Batched drivers: every query's blockers equal the single-query drivers' (and the oracle's)."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2302_13529_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _queries(count=10, seed=7):
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed * 100 + i)
        n = int(rng.integers(300, 6000))
        m = int(n * rng.uniform(3, 10))
        rp, col = W.chung_lu(n, m, 2.1, seed=int(rng.integers(1 << 30)))
        thr = W.wc_thresholds(col, n) if i % 2 == 0 else W.tr_thresholds(len(col), int(rng.integers(1 << 30)))
        g = W.Graph(n, rp, col, thr)
        k = int(rng.integers(1, 40))
        seeds = W.uniform_seeds(n, k, int(rng.integers(1 << 30)))
        b = int(rng.integers(1, 8))
        theta = int(rng.integers(200, 3000))
        out.append((g, seeds, b, theta, int(rng.integers(1 << 62))))
    return out


@pytest.mark.parametrize("driver", ["ag", "gr"])
def test_batch_equals_single_queries(cuda_lib, driver):
    qs = _queries()
    handles = [cuda_lib.load_graph(g) for g, *_ in qs]
    items = [(h, s, b, t, k) for h, (g, s, b, t, k) in zip(handles, qs)]
    batch = (cuda_lib.batch_advanced_greedy if driver == "ag" else cuda_lib.batch_greedy_replace)(items)
    single = cuda_lib.advanced_greedy if driver == "ag" else cuda_lib.greedy_replace
    orc = O.advanced_greedy if driver == "ag" else O.greedy_replace
    for i, ((g, s, b, t, k), h) in enumerate(zip(qs, handles)):
        alone = single(h, s, b, t, k)
        assert np.array_equal(batch[i], alone), (driver, i)
        if i < 4:
            assert np.array_equal(batch[i], orc(g, s, b, t, k)), (driver, i)


def test_batch_edge_cases_and_fallbacks(cuda_lib, monkeypatch):
    g = W.graph_from_edges(6, [(0, 1, 1), (1, 2, 1), (2, 3, Fraction(1, 2)), (4, 5, 1)])
    h = cuda_lib.load_graph(g)
    big = W.random_small_graph(300_000, 600_000, seed=3, p_choices=(Fraction(1, 2), 1))
    hb = cuda_lib.load_graph(big)
    sb = W.uniform_seeds(big.n, 20, 9)
    items = [(h, [5], 3, 100, 1),        # GR: no out-neighbours -> 0 blockers
             (h, [0], 0, 100, 2),        # b = 0
             (h, [0, 1, 2], 10, 50, 3)]  # AG runs out of candidates
    for drv, single in (("ag", cuda_lib.advanced_greedy), ("gr", cuda_lib.greedy_replace)):
        f = cuda_lib.batch_advanced_greedy if drv == "ag" else cuda_lib.batch_greedy_replace
        res = f(items)
        for it, r in zip(items, res):
            assert np.array_equal(r, single(*it)), (drv, it)
        # a graph above 2^18 vertices joins the batch in the global-bitmap size class
        res = f(items + [(hb, sb, 3, 500, 77)])
        assert np.array_equal(res[-1], single(hb, sb, 3, 500, 77))
    # force the batched whole-graph kernel (tiny non-tree capacity in the block tier)
    qs = _queries(4, seed=11)
    hs = [cuda_lib.load_graph(q[0]) for q in qs]
    items = [(hh, s, b, t, k) for hh, (g, s, b, t, k) in zip(hs, qs)]
    want = [cuda_lib.advanced_greedy(*it) for it in items]
    monkeypatch.setenv("IMIN_CTA_EDGE_CAP", "1")
    got = cuda_lib.batch_advanced_greedy(items)
    st = cuda_lib.last_stats()
    monkeypatch.delenv("IMIN_CTA_EDGE_CAP")
    for a, b_ in zip(got, want):
        assert np.array_equal(a, b_)
    assert st["samples"] > 0


@pytest.mark.parametrize("cutoff", ["0", "32", "400"])
def test_batch_warp_block_cutoff(cuda_lib, monkeypatch, cutoff):
    """The batched warp tier finishes the samples within the cutoff and marks them; the block
    launches skip exactly those. Every cutoff (0 = block tier only) gives the single-query result,
    and a query with more seeds than the warp tier holds goes to the block tier alone."""
    qs = _queries(6, seed=23)
    hs = [cuda_lib.load_graph(q[0]) for q in qs]
    items = [(hh, s, b, t, k) for hh, (g, s, b, t, k) in zip(hs, qs)]
    rp, col = W.chung_lu(3000, 20000, 2.1, seed=24)
    gm = W.Graph(3000, rp, col, W.wc_thresholds(col, 3000))
    hm = cuda_lib.load_graph(gm)
    items.append((hm, W.uniform_seeds(3000, 300, 25), 3, 800, 26))  # 300 seeds > warp-tier limit
    want = [cuda_lib.advanced_greedy(*it) for it in items]
    monkeypatch.setenv("IMIN_TIER0_VERTICES", cutoff)
    for f, single in ((cuda_lib.batch_advanced_greedy, None), (cuda_lib.batch_greedy_replace, cuda_lib.greedy_replace)):
        got = f(items)
        st = cuda_lib.last_stats()
        ref = want if single is None else [single(*it) for it in items]
        for i, (a, b_) in enumerate(zip(got, ref)):
            assert np.array_equal(a, b_), (cutoff, i)
        if cutoff == "0":
            assert st["tier_samples"][0] == 0
        else:
            assert st["tier_samples"][0] > 0 and st["tier_samples"][3] > 0, st


def test_batch_queue_granularity_tuning(cuda_lib, monkeypatch):
    """imin_autotune_batch picks one of its candidates, leaves the callers' outputs alone, and the
    batch keeps giving the single-query results with the tuned and with forced granularities."""
    qs = _queries(8, seed=31)
    hs = [cuda_lib.load_graph(q[0]) for q in qs]
    outs = [np.full(max(b, 1), -7, np.int32) for (g, s, b, t, k) in qs]
    items = [(hh, s, b, t, k, o) for hh, (g, s, b, t, k), o in zip(hs, qs, outs)]
    c = cuda_lib.autotune_batch(items, 1)
    assert c in (4, 8, 16, 32, 64)
    assert all((o == -7).all() for o in outs)
    want = [cuda_lib.greedy_replace(*it[:5]) for it in items]
    for forced in (None, "1", "3", "1000"):
        if forced:
            monkeypatch.setenv("IMIN_BATCH_CHUNK", forced)
        got = cuda_lib.batch_greedy_replace([it[:5] for it in items])
        assert all(np.array_equal(a, b) for a, b in zip(got, want)), forced
