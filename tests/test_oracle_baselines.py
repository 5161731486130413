"""Pins of the oracle's comparison algorithms (Sec. 5): BaselineGreedy with simulations (Alg. 1),
Exact, OutDegree, Rand, and the simulated spread of many blocker sets they rest on.

* On every sampled graph, blocking u removes exactly the vertices u dominates (Cor. 1, Thm. 6):
  |R(B)| - |R(B u {u})| = c[u]. With the same samples for every candidate, BaselineGreedy's
  simulated decrease of u in round i is therefore Alg. 2's counter of round i, and BaselineGreedy
  must return AdvancedGreedy's list exactly -- two code paths (BFS reach counts versus
  Lengauer-Tarjan subtree sizes) that share nothing but the random stream.
* Exact against the toy graph's printed optimum (Table 3, Thm. 2) and against brute force over
  all subsets on certain-edge graphs, where every simulation is exact.
* The spread of blocker sets against an independent BFS over each sample's live edges.
* OutDegree on a hand-made graph; Rand against a restatement over the KAT-pinned Philox words.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2302_13529_gb300 import workloads as W
from tests import pins
from tests.test_oracle_pins import TOY


def _small(seed, n=None, certain=False):
    rng = np.random.default_rng(8000 + seed)
    n = n or int(rng.integers(8, 30))
    p = (1,) if certain else (Fraction(1, 2), Fraction(1, 3), Fraction(9, 10), 1)
    g = W.random_small_graph(n, int(rng.integers(n, 3 * n)), seed=8100 + seed, p_choices=p)
    seeds = [int(x) for x in rng.choice(n, int(rng.integers(1, 3)), replace=False)]
    return g, seeds


@pytest.mark.parametrize("seed", range(8))
def test_baseline_greedy_equals_advanced_greedy_on_common_samples(seed):
    g, seeds = _small(seed)
    for b, r in ((1, 50), (3, 200)):
        bg = [int(x) for x in O.baseline_greedy(g, seeds, b, r, 900 + seed)]
        ag = [int(x) for x in O.advanced_greedy(g, seeds, b, r, 900 + seed)]
        assert bg == ag, (seed, b, bg, ag)


def test_baseline_greedy_toy_graph():
    """Table 3: the greedy picks v5 first, then v2 (ties between v2 and v4 go to the smaller id)."""
    assert [int(x) for x in O.baseline_greedy(TOY, [0], 2, 20_000, 3)] == [4, 1]


def test_exact_toy_graph_optimum():
    """b = 1: blocking v5 leaves spread 3 (Ex. 1); b = 2: blocking v2 and v4 isolates the seed
    (spread 1, Table 3)."""
    assert [int(x) for x in O.exact(TOY, [0], 1, 5000, 8)] == [4]
    assert [int(x) for x in O.exact(TOY, [0], 2, 5000, 8)] == [1, 3]


@pytest.mark.parametrize("seed", range(6))
def test_exact_against_brute_force_on_certain_graphs(seed):
    g, seeds = _small(seed, n=11, certain=True)
    live = [(u, int(v)) for u in range(g.n) for v in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]]
    cands = [v for v in range(g.n) if v not in seeds]
    for b in (1, 2, 3):
        best, best_set = None, None
        for sub in itertools.combinations(cands, b):  # lexicographic, first minimum kept
            sp = len(pins.reach(g.n, live, seeds, sub))
            if best is None or sp < best:
                best, best_set = sp, list(sub)
        assert [int(x) for x in O.exact(g, seeds, b, 3, seed)] == best_set, (seed, b)


@pytest.mark.parametrize("seed", range(4))
def test_spread_sets_against_independent_bfs(seed):
    g, seeds = _small(seed)
    rng = np.random.default_rng(seed)
    rest = [v for v in range(g.n) if v not in seeds]
    base = [int(rng.choice(rest))]
    others = [v for v in rest if v not in base]
    sets = [[int(x) for x in rng.choice(others, 2, replace=False)] for _ in range(5)]
    key, rnd, theta = 31 + seed, 4, 40
    got = O.spread_sets(g, seeds, base, sets, theta, key, rnd)
    for s, val in zip(sets, got):
        want = sum(len(pins.reach(g.n, pins.sample_live_edges(g, key, rnd, j, O.edge_word), seeds, base + s))
                   for j in range(theta))
        assert int(val) == want


def test_out_degree_hand_example():
    # out-degrees: 0:3, 1:1, 2:3, 3:0, 4:2, 5:3 ; seed 0
    edges = [(0, 1, 1), (0, 2, 1), (0, 3, 1), (1, 2, 1), (2, 3, 1), (2, 4, 1), (2, 5, 1), (4, 0, 1),
             (4, 1, 1), (5, 0, 1), (5, 1, 1), (5, 2, 1)]
    g = W.graph_from_edges(6, edges)
    assert [int(x) for x in O.out_degree_blockers(g, [0], 4)] == [2, 5, 4, 1]
    assert [int(x) for x in O.out_degree_blockers(g, [0], 10)] == [2, 5, 4, 1, 3]


def test_random_blockers_restated_and_uniform():
    n, seeds = 50, [3, 17]
    for key in (1, 2, 0xFFFFFFFFFFFF):
        cand = [u for u in range(n) if u not in seeds]
        want = []
        for t in range(7):
            w = int(O.philox4x32_10([t, 0, 0, 0xC0000000], [key & 0xFFFFFFFF, key >> 32])[0])
            pick = t + ((w * (len(cand) - t)) >> 32)
            cand[t], cand[pick] = cand[pick], cand[t]
            want.append(cand[t])
        assert [int(x) for x in O.random_blockers(n, seeds, 7, key)] == want
    firsts = np.bincount([int(O.random_blockers(10, [0], 1, k)[0]) for k in range(9000)], minlength=10)
    assert firsts[0] == 0 and all(abs(c - 1000) < 150 for c in firsts[1:])
    assert len(O.random_blockers(5, [0, 1], 10, 3)) == 3
