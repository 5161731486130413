"""Serving: requests submitted at different times share batched steps; every result must equal
the single-query driver's result for the same request (and the oracle's)."""
from __future__ import annotations

import time
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2302_13529_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _graphs():
    g1 = W.tiny_chung_lu_query().graph
    rp, col = W.chung_lu(30_000, 240_000, 2.1, seed=5)
    g2 = W.Graph(30_000, rp, col, W.tr_thresholds(len(col), 6))
    g3 = W.graph_rmat_wc(12, 30_000, seed=7)
    return [g1, g2, g3]


def _requests(graphs, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        gi = int(rng.integers(0, len(graphs)))
        g = graphs[gi]
        k = int(rng.integers(1, 40))
        out.append(dict(driver=int(rng.integers(0, 2)), gi=gi,
                        seeds=W.uniform_seeds(g.n, k, int(rng.integers(1 << 30))),
                        b=int(rng.integers(0, 8)), theta=int(rng.integers(300, 4000)),
                        key=int(rng.integers(1 << 62))))
    return out


def _alone(cuda_lib, hs, r):
    f = cuda_lib.advanced_greedy if r["driver"] == 0 else cuda_lib.greedy_replace
    return f(hs[r["gi"]], r["seeds"], r["b"], r["theta"], r["key"])


@pytest.mark.parametrize("max_active,budget", [(5, 0), (64, 0), (8, 3 << 20)])
def test_results_in_the_mix_equal_results_alone(cuda_lib, max_active, budget):
    graphs = _graphs()
    hs = [cuda_lib.load_graph(g) for g in graphs]
    reqs = _requests(graphs, 18, seed=max_active)
    want = [_alone(cuda_lib, hs, r) for r in reqs]
    with cuda_lib.Server(memory_budget=budget, max_active=max_active) as srv:
        tickets = []
        for i, r in enumerate(reqs):  # arrivals spread over time: later ones join running steps
            tickets.append(srv.submit(r["driver"], hs[r["gi"]], r["seeds"], r["b"], r["theta"], r["key"]))
            if i % 5 == 4:
                time.sleep(0.01)
        got = [srv.wait(t, capacity=max(r["b"], 1))[0] for t, r in zip(tickets, reqs)]
        st = srv.stats()
    for i, (a, b) in enumerate(zip(got, want)):
        assert np.array_equal(a, b), (i, reqs[i])
    assert st["completed"] == len(reqs) and st["memory_in_use"] == 0
    for r, g in zip(reqs[:3], got[:3]):
        f = O.advanced_greedy if r["driver"] == 0 else O.greedy_replace
        assert np.array_equal(g, f(graphs[r["gi"]], r["seeds"], r["b"], r["theta"], r["key"]))


def test_serving_large_graph_and_errors(cuda_lib):
    from paper_2302_13529_gb300.imin import IminError
    big = W.graph_rmat_wc(19, 1 << 20, seed=91)
    small = W.tiny_chung_lu_query()
    hb, hs = cuda_lib.load_graph(big), cuda_lib.load_graph(small.graph)
    sb = W.uniform_seeds(big.n, 30, 92)
    with cuda_lib.Server(max_active=4) as srv:
        t1 = srv.submit(0, hb, sb, 3, 1500, 94)
        t2 = srv.submit(1, hs, small.seeds, 4, 2000, small.key)
        t3 = srv.submit(0, hs, small.seeds, 6, 200_000, 5)  # long enough not to be done at once
        with pytest.raises(IminError) as e:
            srv.wait(t3, capacity=6, timeout_ms=0)
        assert e.value.code == -6
        with pytest.raises(IminError):
            srv.submit(0, hs, [0, 0], 2, 100, 1)  # duplicate seed
        b1, lat1 = srv.wait(t1, capacity=3)
        b2, _ = srv.wait(t2, capacity=4)
        b3, _ = srv.wait(t3, capacity=6)
        with pytest.raises(IminError):
            srv.wait(t1, capacity=3)  # already collected
    assert np.array_equal(b1, cuda_lib.advanced_greedy(hb, sb, 3, 1500, 94))
    assert np.array_equal(b2, cuda_lib.greedy_replace(hs, small.seeds, 4, 2000, small.key))
    assert np.array_equal(b3, cuda_lib.advanced_greedy(hs, small.seeds, 6, 200_000, 5))
    assert lat1 > 0


def test_serving_mixes_warp_tier_and_block_only_requests(cuda_lib):
    """A request whose seed set is too large for the warp tier (300 seeds) runs next to small ones;
    the warp tier serves only the small ones, and every result equals the request run alone."""
    graphs = _graphs()
    hs = [cuda_lib.load_graph(g) for g in graphs]
    reqs = _requests(graphs, 6, seed=77)
    reqs.append(dict(driver=1, gi=1, seeds=W.uniform_seeds(graphs[1].n, 300, 78), b=4, theta=1500, key=79))
    reqs.append(dict(driver=0, gi=2, seeds=W.uniform_seeds(graphs[2].n, 280, 80), b=3, theta=900, key=81))
    want = [_alone(cuda_lib, hs, r) for r in reqs]
    with cuda_lib.Server(max_active=16) as srv:
        tickets = [srv.submit(r["driver"], hs[r["gi"]], r["seeds"], r["b"], r["theta"], r["key"]) for r in reqs]
        got = [srv.wait(t, capacity=max(r["b"], 1))[0] for t, r in zip(tickets, reqs)]
    for i, (a, b) in enumerate(zip(got, want)):
        assert np.array_equal(a, b), (i, reqs[i]["b"], len(reqs[i]["seeds"]))


@pytest.mark.parametrize("class_cap", [0, 1])
def test_size_classes_take_turns(cuda_lib, class_cap):
    """Requests on graphs of three size classes (n = 2,000, 2^17 and 2^19: the last with the
    visited bitmap in global memory) arrive while others run. Each step serves one class, so a
    request sits out the steps of the other classes; its rounds, random streams and result must
    still be exactly those of the request run alone. With a per-class cap of one sampled graph per
    step, each class runs one request at a time and admission passes over a class at its cap."""
    graphs = [W.tiny_chung_lu_query().graph, W.graph_rmat_wc(17, 1 << 19, seed=41),
              W.graph_rmat_wc(19, 1 << 20, seed=91)]
    hs = [cuda_lib.load_graph(g) for g in graphs]
    rng = np.random.default_rng(43)
    reqs = []
    for i in range(9):
        gi = i % 3
        g = graphs[gi]
        reqs.append(dict(driver=int(i % 2), gi=gi, seeds=W.uniform_seeds(g.n, int(rng.integers(5, 40)), 100 + i),
                         b=int(rng.integers(2, 7)), theta=int(rng.integers(500, 3000)), key=int(rng.integers(1 << 62))))
    want = [_alone(cuda_lib, hs, r) for r in reqs]
    with cuda_lib.Server(max_active=8, max_class_samples=class_cap) as srv:
        tickets = []
        for i, r in enumerate(reqs):
            tickets.append(srv.submit(r["driver"], hs[r["gi"]], r["seeds"], r["b"], r["theta"], r["key"]))
            if i % 3 == 2:
                time.sleep(0.02)
        got = [srv.wait(t, capacity=r["b"])[0] for t, r in zip(tickets, reqs)]
        st = srv.stats()
    for i, (a, b) in enumerate(zip(got, want)):
        assert np.array_equal(a, b), (i, reqs[i]["gi"], reqs[i]["driver"])
    assert st["completed"] == len(reqs) and st["memory_in_use"] == 0
    r = reqs[1]  # the 2^17 graph: one result against the oracle as well
    f = O.advanced_greedy if r["driver"] == 0 else O.greedy_replace
    assert np.array_equal(got[1], f(graphs[1], r["seeds"], r["b"], r["theta"], r["key"]))
