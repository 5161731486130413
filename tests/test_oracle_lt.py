"""Pins of the oracle's linear-threshold (LT) model, the standard triggering model (Sec. 4.5:
every vertex draws a triggering set of in-neighbours and only edges from it stay; under LT the
set holds at most one in-neighbour u, with probability b(u, v)). Each check is independent of the
oracle's own sampling code: exact enumeration of all triggering worlds, per-sample brute force on
live edges rebuilt from the KAT-pinned Philox stream, and a case that reduces to the IC model."""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2302_13529_gb300 import workloads as W
from tests import pins


def _lt_graph(n, m, seed, certain_frac=0.0):
    """A random simple graph with LT shares: each vertex's in-edges split a random total <= 1."""
    rng = np.random.default_rng(seed)
    g = W.random_small_graph(n, m, seed=seed, p_choices=(1,))
    thr = np.zeros(len(g.col), dtype=np.uint32)
    for v in range(n):
        es = np.nonzero(g.col == v)[0]
        if len(es) == 0:
            continue
        total = 1.0 if rng.random() < certain_frac else rng.uniform(0.3, 1.0)
        w = rng.dirichlet(np.ones(len(es))) * total
        shares = np.maximum(1, np.floor(w * W.TWO32)).astype(np.uint64)
        while shares.sum() > W.TWO32:
            shares[np.argmax(shares)] -= shares.sum() - W.TWO32
        thr[es] = (shares - 1).astype(np.uint32)
    return W.Graph(n, g.row_ptr, g.col, thr)


def test_vertex_word_layout_and_separation():
    """A vertex word is one word of the KAT-pinned Philox stream under its own last counter word,
    so it never coincides with the edge-word stream."""
    key = 0x0123456789ABCDEF
    for v in (0, 1, 2, 3, 4, 1001, 2 ** 30 + 5):
        ctr = [v >> 2, 7, 3, 0x80000000]
        want = O.philox4x32_10(ctr, [key & 0xFFFFFFFF, key >> 32])[v & 3]
        assert O.vertex_word(key, 3, 7, v) == int(want)
    assert [O.vertex_word(5, 0, 0, v) for v in range(8)] != [O.edge_word(5, 0, 0, e) for e in range(8)]


@pytest.mark.parametrize("seed", range(8))
def test_lt_sample_matches_vertex_deletion(seed):
    """Every LT sample keeps at most one in-edge per vertex, and the oracle's subtree sizes and
    dominators equal brute force by vertex deletion on the rebuilt live edges."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(6, 30))
    g = _lt_graph(n, int(rng.integers(n, 3 * n)), seed=200 + seed)
    seeds = [int(x) for x in rng.choice(n, 2, replace=False)]
    rest = [v for v in range(n) if v not in seeds]
    blocked = [int(rng.choice(rest))]
    key, rnd = 4000 + seed, 2
    for j in range(12):
        live = pins.lt_sample_live_edges(g, key, rnd, j, O.vertex_word)
        indeg = np.bincount([v for _, v in live], minlength=n)
        assert indeg.max(initial=0) <= 1
        R, c_want, idom_want = pins.brute_force_sample(g, seeds, blocked, live)
        c, idom, nr, _ = O.sample(g, seeds, blocked, key, rnd, j, model="lt")
        assert nr == len(R)
        assert (c.astype(np.int64) == c_want).all(), (seed, j)
        for v in R:
            if v not in seeds:
                assert idom[v] == idom_want[v], (seed, j, v)


@pytest.mark.parametrize("seed", range(5))
def test_lt_estimator_and_spread_against_enumeration(seed):
    rng = np.random.default_rng(300 + seed)
    n = 7
    g = _lt_graph(n, 12, seed=400 + seed)
    seeds = [int(x) for x in rng.choice(n, 2, replace=False)]
    try:
        spread, dec, dec2 = pins.exact_lt_moments(g, seeds)
    except ValueError:
        pytest.skip("too many worlds")
    theta = 40_000
    got = O.decrease(g, seeds, [], theta, key=77 + seed, model="lt").astype(np.float64) / theta
    for u in range(n):
        if u in seeds:
            assert got[u] == 0
            continue
        sd = math.sqrt(max(dec2[u] - dec[u] ** 2, 0.0) / theta)
        assert abs(got[u] - dec[u]) <= 6 * sd + 1e-9, (u, got[u], dec[u], sd)
    # the spread: |R| per sample is at most n, so sd <= n / (2 sqrt(theta))
    s = O.spread(g, seeds, [], theta, key=88 + seed, model="lt") / theta
    assert abs(s - spread) <= 6 * n / (2 * math.sqrt(theta)), (s, spread)


def test_lt_with_single_certain_in_edges_is_ic_with_p1():
    """When every vertex has at most one in-edge and it holds the whole share, the LT sample is
    the graph itself, as is the IC sample with p = 1: the two models agree exactly."""
    rng = np.random.default_rng(9)
    n = 60
    parent = [-1] + [int(rng.integers(0, v)) for v in range(1, n)]  # a random out-tree
    edges = [(parent[v], v, 1) for v in range(1, n)]
    g = W.graph_from_edges(n, edges)
    assert np.all(g.thr == 0xFFFFFFFF)
    for seeds, blocked in (([0], []), ([0, 5], [7])):
        a = O.decrease(g, seeds, blocked, 50, 3, model="lt")
        b = O.decrease(g, seeds, blocked, 50, 3, model="ic")
        assert np.array_equal(a, b)
        assert O.spread(g, seeds, blocked, 50, 3, model="lt") == O.spread(g, seeds, blocked, 50, 3)


def test_lt_rejects_shares_above_one():
    g = W.graph_from_edges(3, [(0, 2, Fraction(3, 4)), (1, 2, Fraction(1, 2))])
    with pytest.raises(ValueError):
        O.decrease(g, [0], [], 10, 1, model="lt")
    with pytest.raises(ValueError):
        O.decrease(g, [0], [], 10, 1, model="xx")


def test_lt_wc_weights_fill_but_never_exceed_one():
    rp, col = W.chung_lu(2000, 9000, 2.1, seed=8)
    t = W.lt_wc_weights(col, 2000)
    acc = np.zeros(2000, dtype=np.uint64)
    np.add.at(acc, col, t.astype(np.uint64) + 1)
    d = np.bincount(col, minlength=2000)
    assert np.all(acc <= W.TWO32)
    assert np.all(W.TWO32 - acc[d > 0] < d[d > 0])  # at most d - 1 units of 2^-32 left unused


def test_lt_advanced_greedy_first_pick_is_the_exact_argmax():
    """With theta large, AdvancedGreedy's first LT blocker is the exact expected-decrease argmax
    whenever the runner-up trails by more than 8 standard deviations."""
    checked = 0
    for seed in range(12):
        rng = np.random.default_rng(500 + seed)
        g = _lt_graph(8, 14, seed=600 + seed, certain_frac=0.5)
        seeds = [int(rng.integers(0, 8))]
        try:
            _, dec, dec2 = pins.exact_lt_moments(g, seeds)
        except ValueError:
            continue
        theta = 20_000
        order = [u for u in np.argsort(-dec, kind="stable") if u not in seeds]
        best, second = order[0], order[1]
        sd = math.sqrt((max(dec2[best] - dec[best] ** 2, 0) + max(dec2[second] - dec[second] ** 2, 0)) / theta)
        if dec[best] - dec[second] <= 8 * sd:
            continue
        B = O.advanced_greedy(g, seeds, 1, theta, 900 + seed, model="lt")
        assert int(B[0]) == int(best), (seed, dec)
        checked += 1
    assert checked >= 3
