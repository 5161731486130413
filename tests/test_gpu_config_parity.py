"""Bit-exact parity with the oracle at the sizes of the five measured workloads.

Every arithmetic step on the path is integer, so counters and blocker lists must be identical.
The random stream is counter-based: any Alg. 2 call of a greedy run can be replayed on its own
from the GPU's blocker prefix (round r sees B[:r]), which is how the workloads too large for a
full oracle run are checked. The oracle runs on all host cores (tests/oracle_pool.py); its
sample loop splits into independent integer sums, so the result is the sequential one.

What each test replays is stated in its docstring:
  * R-MAT 2^17 / 2^20, WC, |S| = 50, b = 50, theta = 10^5: AdvancedGreedy and GreedyReplace in
    full (every round of both phases, and where GreedyReplace stops);
  * 256 Chung-Lu TR queries in one batch: 8 queries in full, among them the largest n and the
    largest |S|, and 3 GreedyReplace queries;
  * R-MAT 2^22 / 2^26, WC, |S| = 200: 20,000 samples of round 0 and of round 150 of the full
    AdvancedGreedy run (b = 200, theta = 2*10^5), plus AdvancedGreedy and GreedyReplace in full
    at b = 3, theta = 2,000 on the same graph and seeds;
  * serving: 2 requests on each graph from the serving request mix, run in one server next to
    each other; the R-MAT 2^17 requests are replayed in full, the R-MAT 2^22 ones in their first
    and last rounds (full theta).
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2302_13529_gb300 import workloads as W
from tests import oracle_pool
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _argmax(d, excluded):
    """Strict '>' in ascending id over the vertices not excluded (smallest id among the maxima)."""
    d = d.astype(np.int64)
    d[np.asarray(list(excluded), dtype=np.int64)] = -1
    return int(np.argmax(d))


# --------------------------------------------------------------------------------------------
# R-MAT 2^17 / 2^20 (mid-scale single query)
# --------------------------------------------------------------------------------------------

def test_rmat17_advanced_greedy_every_round(cuda_lib):
    """All 50 rounds of AdvancedGreedy at full size (5*10^6 sampled graphs): the GPU's list equals
    the oracle's, element by element."""
    q = W.rmat17_query()
    gh = cuda_lib.load_graph(q.graph)
    got = [int(x) for x in cuda_lib.advanced_greedy(gh, q.seeds, q.b, q.theta, q.key)]
    st = cuda_lib.last_stats()
    want = [int(x) for x in oracle_pool.advanced_greedy(q.graph, q.seeds, q.b, q.theta, q.key)]
    assert got == want
    assert st["samples"] == q.b * q.theta


def test_rmat17_greedy_replace_every_round(cuda_lib):
    """GreedyReplace at full size: every phase-1 call, every phase-2 call and the early stop. The
    lists must be equal, and the GPU must have sampled exactly as many graphs as the oracle's
    calls up to its stop (theta per call)."""
    q = W.rmat17_query()
    gh = cuda_lib.load_graph(q.graph)
    got = [int(x) for x in cuda_lib.greedy_replace(gh, q.seeds, q.b, q.theta, q.key)]
    st = cuda_lib.last_stats()
    want = [int(x) for x in oracle_pool.greedy_replace(q.graph, q.seeds, q.b, q.theta, q.key)]
    calls = O.last_calls()
    assert got == want
    assert st["samples"] == calls * q.theta, (st["samples"], calls)
    assert q.b < calls <= 2 * q.b


# --------------------------------------------------------------------------------------------
# 256 Chung-Lu TR queries, one batched call
# --------------------------------------------------------------------------------------------

def _batch_subset(qs):
    ns = [q.graph.n for q in qs]
    ks = [len(q.seeds) for q in qs]
    ms = [q.graph.m for q in qs]
    pick = [int(np.argmax(ns)), int(np.argmax(ks)), int(np.argmax(ms)), int(np.argmin(ns)),
            int(np.argmin(ks))]
    for i in range(0, len(qs), 37):
        if len(set(pick)) >= 8:
            break
        pick.append(i)
    return sorted(set(pick))


def test_batch256_queries_against_oracle(cuda_lib):
    """The 256-query batch at its configured sizes (n log-uniform in [10^3, 2*10^5], TR, b = 20,
    theta = 2*10^4): 8 queries -- largest n, largest |S|, largest m, smallest n, smallest |S| and
    every 37th -- replayed by the oracle in full; then the same batch under GreedyReplace with 3
    of those queries replayed."""
    qs = W.batch_queries(256)
    hs = [cuda_lib.load_graph(q.graph) for q in qs]
    items = [(h, q.seeds, q.b, q.theta, q.key) for h, q in zip(hs, qs)]
    ag = cuda_lib.batch_advanced_greedy(items)
    chosen = _batch_subset(qs)
    assert len(chosen) >= 8
    for i in chosen:
        q = qs[i]
        want = [int(x) for x in oracle_pool.advanced_greedy(q.graph, q.seeds, q.b, q.theta, q.key)]
        assert [int(x) for x in ag[i]] == want, (i, q.graph.n, len(q.seeds))
    gr = cuda_lib.batch_greedy_replace(items)
    for i in chosen[:3]:
        q = qs[i]
        want = [int(x) for x in oracle_pool.greedy_replace(q.graph, q.seeds, q.b, q.theta, q.key)]
        assert [int(x) for x in gr[i]] == want, i


# --------------------------------------------------------------------------------------------
# R-MAT 2^22 / 2^26 (large single query)
# --------------------------------------------------------------------------------------------

def test_rmat22_rounds_from_gpu_prefix(cuda_lib):
    """The full AdvancedGreedy run (b = 200, theta = 2*10^5) on the GPU; then the first 20,000
    sampled graphs of round 0 and of round 150 (blocked: the GPU's first 150 blockers), every
    counter against the oracle."""
    q = W.rmat22_query()
    gh = cuda_lib.load_graph(q.graph)
    B = cuda_lib.advanced_greedy(gh, q.seeds, q.b, q.theta, q.key)
    assert len(B) == q.b and len(set(B.tolist())) == q.b and not set(B.tolist()) & set(q.seeds.tolist())
    for r in (0, 150):
        got = cuda_lib.estimate_decrease(gh, q.seeds, B[:r], 20_000, q.key, r)
        want = oracle_pool.decrease(q.graph, q.seeds, B[:r], 20_000, q.key, r)
        assert np.array_equal(got, want), r


def test_rmat22_small_budget_drivers(cuda_lib):
    """The large graph and its 200 seeds with b = 3 and theta = 2,000: AdvancedGreedy and
    GreedyReplace in full against the oracle."""
    q = W.rmat22_query()
    gh = cuda_lib.load_graph(q.graph)
    for f, o in ((cuda_lib.advanced_greedy, oracle_pool.advanced_greedy),
                 (cuda_lib.greedy_replace, oracle_pool.greedy_replace)):
        got = [int(x) for x in f(gh, q.seeds, 3, 2000, q.key)]
        want = [int(x) for x in o(q.graph, q.seeds, 3, 2000, q.key)]
        assert got == want, f.__name__


# --------------------------------------------------------------------------------------------
# serving mix on the R-MAT 2^17 and 2^22 graphs
# --------------------------------------------------------------------------------------------

def test_serving_requests_against_oracle(cuda_lib):
    """The first 30 requests of the serving mix; on each graph the 2 with the fewest sampled
    graphs (b * theta * |S|), served together in one server. R-MAT 2^17 requests: the oracle
    replays every round. R-MAT 2^22 requests: rounds 0 and b-1 in full (theta samples each), whose
    argmax given the served prefix must be the served blocker."""
    reqs = W.serving_requests(30)
    graphs = [W.rmat17_query().graph, W.rmat22_query().graph]
    hs = [cuda_lib.load_graph(g) for g in graphs]
    chosen = []
    for gi in (0, 1):
        idx = [i for i, r in enumerate(reqs) if r.gi == gi]
        idx.sort(key=lambda i: reqs[i].b * reqs[i].theta * len(reqs[i].seeds))
        chosen += idx[:2]
    with cuda_lib.Server(max_active=8) as srv:
        tickets = [srv.submit(0, hs[reqs[i].gi], reqs[i].seeds, reqs[i].b, reqs[i].theta, reqs[i].key)
                   for i in chosen]
        served = [srv.wait(t, capacity=reqs[i].b)[0] for t, i in zip(tickets, chosen)]
    for i, B in zip(chosen, served):
        r = reqs[i]
        g = graphs[r.gi]
        B = [int(x) for x in B]
        assert len(B) == r.b
        if r.gi == 0:
            assert B == [int(x) for x in oracle_pool.advanced_greedy(g, r.seeds, r.b, r.theta, r.key)], i
        else:
            for k in (0, r.b - 1):
                d = oracle_pool.decrease(g, r.seeds, B[:k], r.theta, r.key, k)
                assert _argmax(d, set(r.seeds.tolist()) | set(B[:k])) == B[k], (i, k)
