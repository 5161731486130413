"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle, bit for bit.

All arithmetic on the path is integer (Philox words, threshold compares, subtree sizes and
uint64 sums), so the tolerance is zero: counters and blockers must be identical.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2302_13529_gb300 import workloads as W
from tests import oracle_pool

pytestmark = pytest.mark.gpu


def _small_case(i):
    rng = np.random.default_rng(1000 + i)
    n = int(rng.integers(5, 40))
    m = int(rng.integers(n, 4 * n))
    g = W.random_small_graph(n, m, seed=2000 + i)
    k = int(rng.integers(1, min(5, n)))
    seeds = [int(x) for x in rng.choice(n, k, replace=False)]
    rest = [v for v in range(n) if v not in seeds]
    nb = int(rng.integers(0, min(4, len(rest)) + 1))
    blocked = [int(x) for x in rng.choice(rest, nb, replace=False)] if nb else []
    return g, seeds, blocked


@pytest.mark.parametrize("i", range(16))
def test_decrease_small_graphs(cuda_lib, i):
    g, seeds, blocked = _small_case(i)
    gh = cuda_lib.load_graph(g)
    for theta, key, rnd in ((1, 5, 0), (37, 77, 3), (2000, 0xDEADBEEFCAFE, 11)):
        want = O.decrease(g, seeds, blocked, theta, key, rnd)
        got = cuda_lib.estimate_decrease(gh, seeds, blocked, theta, key, rnd)
        assert np.array_equal(got, want), (i, theta)


def test_toy_graph_counters(cuda_lib):
    from tests.test_oracle_pins import TOY
    gh = cuda_lib.load_graph(TOY)
    for key in (1, 99):
        want = O.decrease(TOY, [0], [], 50_000, key)
        got = cuda_lib.estimate_decrease(gh, [0], [], 50_000, key)
        assert np.array_equal(got, want)
    assert list(cuda_lib.advanced_greedy(gh, [0], 2, 20_000, 3)) == [4, 1]
    assert list(cuda_lib.greedy_replace(gh, [0], 2, 20_000, 3)) == [1, 3]
    assert list(cuda_lib.greedy_replace(gh, [0], 1, 20_000, 3)) == [4]


def test_hand_worked_greedy_replace_lists(cuda_lib):
    """The certain-edge graphs whose AdvancedGreedy / GreedyReplace lists are worked out by hand
    (list order, the slot of a replacement, the reverse walk and the early stop of Alg. 4), and
    the number of sampled graphs each run took (theta per Alg. 2 call up to the stop)."""
    from tests.test_oracle_greedy_replace import GOLDEN_CASES
    for name, g, seeds, want in GOLDEN_CASES:
        gh = cuda_lib.load_graph(g)
        for alg, b, lst, calls in want:
            f = cuda_lib.greedy_replace if alg == "GR" else cuda_lib.advanced_greedy
            assert [int(x) for x in f(gh, seeds, b, 5, 3)] == lst, (name, alg, b)
            assert cuda_lib.last_stats()["samples"] == 5 * calls, (name, alg, b)


@pytest.fixture(scope="module")
def tiny():
    return W.tiny_chung_lu_query()


def test_decrease_chung_lu(cuda_lib, tiny):
    q = tiny
    gh = cuda_lib.load_graph(q.graph)
    blocked = [int(x) for x in np.setdiff1d(np.arange(60), q.seeds)[:7]]
    for rnd, bl in ((0, []), (4, blocked)):
        want = O.decrease(q.graph, q.seeds, bl, q.theta, q.key, rnd)
        got, st = cuda_lib.estimate_decrease(gh, q.seeds, bl, q.theta, q.key, rnd, stats=True)
        assert np.array_equal(got, want)
        assert st["samples"] == q.theta


def test_advanced_greedy_chung_lu(cuda_lib, tiny):
    q = tiny
    gh = cuda_lib.load_graph(q.graph)
    want = O.advanced_greedy(q.graph, q.seeds, q.b, q.theta, q.key)
    got = cuda_lib.advanced_greedy(gh, q.seeds, q.b, q.theta, q.key)
    assert np.array_equal(got, want)


def test_greedy_replace_chung_lu(cuda_lib, tiny):
    q = tiny
    gh = cuda_lib.load_graph(q.graph)
    want = O.greedy_replace(q.graph, q.seeds, q.b, q.theta, q.key)
    got = cuda_lib.greedy_replace(gh, q.seeds, q.b, q.theta, q.key)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("path", ["warp-tiers", "block-tier-overflow", "warp-then-block"])
def test_tier_fallback_paths(cuda_lib, monkeypatch, path):
    """Tiny capacities push samples through every tier of a pipeline; results must not change.
    warp-tiers: shared-memory hash -> 16K global scratch -> whole-graph scratch;
    block-tier-overflow: block-per-sample bitmap tier -> whole-graph scratch;
    warp-then-block: warp tier with a 32-vertex cutoff -> block tier -> whole-graph scratch."""
    g = W.graph_rmat_wc(11, 16000, seed=5)
    seeds = W.uniform_seeds(g.n, 12, seed=6)
    want = O.decrease(g, seeds, [], 3000, 1234, 2)
    gh = cuda_lib.load_graph(g)
    if path == "warp-tiers":
        monkeypatch.setenv("IMIN_DISABLE_CTA_TIER", "1")
        monkeypatch.setenv("IMIN_TIER0_VERTICES", "32")
        monkeypatch.setenv("IMIN_TIER1_VERTICES", "64")
        used = (0, 1, 2)
    elif path == "block-tier-overflow":
        monkeypatch.setenv("IMIN_TIER0_VERTICES", "0")
        monkeypatch.setenv("IMIN_CTA_EDGE_CAP", "2")
        used = (3, 2)
    else:
        monkeypatch.setenv("IMIN_TIER0_VERTICES", "32")
        monkeypatch.setenv("IMIN_CTA_EDGE_CAP", "2")
        used = (0, 3, 2)
    got, st = cuda_lib.estimate_decrease(gh, seeds, [], 3000, 1234, 2, stats=True)
    assert np.array_equal(got, want)
    assert all(st["tier_samples"][t] > 0 for t in used), st
    assert sum(st["tier_samples"]) == 3000
    for k in ("IMIN_DISABLE_CTA_TIER", "IMIN_TIER0_VERTICES", "IMIN_TIER1_VERTICES",
              "IMIN_CTA_EDGE_CAP"):
        monkeypatch.delenv(k, raising=False)
    got2, st2 = cuda_lib.estimate_decrease(gh, seeds, [], 3000, 1234, 2, stats=True)
    assert np.array_equal(got2, want)
    # default pipeline for n <= 2^18: the tuned warp/block cutoff, then the block tier
    assert st2["tier_samples"][0] + st2["tier_samples"][3] == 3000


@pytest.mark.parametrize("cutoff", [0, 48, 96, 192, 400])
def test_warp_block_cutoff_does_not_change_counters(cuda_lib, monkeypatch, cutoff):
    """Every warp/block cutoff splits the samples differently between the two kernels; the
    counters and blockers must equal the oracle's for all of them."""
    g = W.graph_rmat_wc(12, 40000, seed=15)
    seeds = W.uniform_seeds(g.n, 20, seed=16)
    monkeypatch.setenv("IMIN_TIER0_VERTICES", str(cutoff))
    gh = cuda_lib.load_graph(g)
    got, st = cuda_lib.estimate_decrease(gh, seeds, [5, 7], 4000, 77, 4, stats=True)
    assert np.array_equal(got, O.decrease(g, seeds, [5, 7], 4000, 77, 4))
    assert sum(st["tier_samples"]) == 4000
    if cutoff == 0:
        assert st["tier_samples"][0] == 0
    else:
        assert st["tier_samples"][0] > 0 and st["tier_samples"][3] > 0, st
    B = cuda_lib.advanced_greedy(gh, seeds, 3, 2000, 78)
    assert np.array_equal(B, O.advanced_greedy(g, seeds, 3, 2000, 78))


def test_autotune(cuda_lib, monkeypatch):
    """imin_autotune picks one of the candidate cutoffs; later calls (which use the cached value)
    still match the oracle; IMIN_AUTOTUNE=0 falls back to the fixed cutoff."""
    g = W.graph_rmat_wc(12, 40000, seed=15)
    seeds = W.uniform_seeds(g.n, 20, seed=16)
    monkeypatch.delenv("IMIN_TIER0_VERTICES", raising=False)
    gh = cuda_lib.load_graph(g)
    c = cuda_lib.autotune(gh, seeds, 99)
    assert c in (0, 64, 96, 128, 192)
    want = O.decrease(g, seeds, [], 3000, 5, 1)
    assert np.array_equal(cuda_lib.estimate_decrease(gh, seeds, [], 3000, 5, 1), want)
    monkeypatch.setenv("IMIN_AUTOTUNE", "0")
    got, st = cuda_lib.estimate_decrease(gh, seeds, [], 3000, 5, 1, stats=True)
    assert np.array_equal(got, want)
    assert st["tier_samples"][0] > 0


def test_warp_tiers_match_on_full_size_round(cuda_lib, monkeypatch, rmat17):
    """The warp-tier pipeline (tiers 0, 1 and 2 without the block tier) and the default pipeline
    on the bench graph, one call at theta = 20,000 each, both against the oracle."""
    q = rmat17
    gh = cuda_lib.load_graph(q.graph)
    want = oracle_pool.decrease(q.graph, q.seeds, [], 20_000, q.key, 3)
    assert np.array_equal(cuda_lib.estimate_decrease(gh, q.seeds, [], 20_000, q.key, 3), want)
    monkeypatch.setenv("IMIN_DISABLE_CTA_TIER", "1")
    assert np.array_equal(cuda_lib.estimate_decrease(gh, q.seeds, [], 20_000, q.key, 3), want)


def test_device_pointers_and_determinism(cuda_lib, tiny):
    import torch
    q = tiny
    gh = cuda_lib.load_graph(q.graph)
    seeds_d = torch.from_numpy(q.seeds).cuda()
    out = torch.zeros(q.graph.n, dtype=torch.uint64, device="cuda")
    cuda_lib.estimate_decrease(gh, seeds_d, None, 5000, q.key, 1, out=out)
    torch.cuda.synchronize()
    want = O.decrease(q.graph, q.seeds, [], 5000, q.key, 1)
    assert np.array_equal(out.cpu().numpy(), want)
    again = cuda_lib.estimate_decrease(gh, q.seeds, [], 5000, q.key, 1)
    assert np.array_equal(again, want)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        third = cuda_lib.estimate_decrease(gh, q.seeds, [], 5000, q.key, 1)
    assert np.array_equal(third, want)
    blk = torch.zeros(q.b, dtype=torch.int32, device="cuda")
    cuda_lib.advanced_greedy(gh, seeds_d, q.b, 2000, q.key, out=blk)
    assert np.array_equal(blk.cpu().numpy(), O.advanced_greedy(q.graph, q.seeds, q.b, 2000, q.key))


def test_edge_cases(cuda_lib):
    g = W.graph_from_edges(6, [(0, 1, 1), (1, 2, 1), (2, 0, 1), (3, 4, W.Fraction(1, 2))])
    gh = cuda_lib.load_graph(g)
    # an isolated seed reaches nothing
    assert not cuda_lib.estimate_decrease(gh, [5], [], 100, 1).any()
    # a cycle back into the seed is ignored
    d = cuda_lib.estimate_decrease(gh, [0], [], 10, 1)
    assert list(d) == [0, 20, 10, 0, 0, 0]
    # every vertex but one is a seed
    d = cuda_lib.estimate_decrease(gh, [0, 1, 2, 3, 4], [], 64, 9)
    assert np.array_equal(d, O.decrease(g, [0, 1, 2, 3, 4], [], 64, 9))
    # AG stops when the candidates run out; GR with no out-neighbours returns nothing
    assert sorted(cuda_lib.advanced_greedy(gh, [0, 1, 2], 10, 20, 1)) == [3, 4, 5]
    assert len(cuda_lib.greedy_replace(gh, [5], 3, 20, 1)) == 0
    assert len(cuda_lib.advanced_greedy(gh, [0], 0, 20, 1)) == 0
    # graph without edges
    g0 = W.Graph(3, np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    gh0 = cuda_lib.load_graph(g0)
    assert not cuda_lib.estimate_decrease(gh0, [1], [], 5, 1).any()


def test_invalid_arguments(cuda_lib):
    from paper_2302_13529_gb300.imin import IminError
    g = W.graph_from_edges(4, [(0, 1, 1), (1, 2, 1)])
    gh = cuda_lib.load_graph(g)
    for seeds, blocked in (([0, 0], []), ([0], [0]), ([4], []), ([0], [1, 1]), ([-1], [])):
        with pytest.raises(IminError) as e:
            cuda_lib.estimate_decrease(gh, seeds, blocked, 10, 1)
        assert e.value.code == -1
    with pytest.raises(IminError):
        cuda_lib.estimate_decrease(gh, [0], [], 0, 1)
    with pytest.raises(IminError):
        cuda_lib.GraphHandle(3, np.array([0, 1, 0, 1], np.int32), np.array([1], np.int32),
                             np.array([5], np.uint32))


# --------------------------------------------------------------------------------------------
# full-size workload: R-MAT 2^17 / 2^20, WC, |S| = 50, theta = 10^5 (bench configuration)
# --------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def rmat17():
    return W.rmat17_query()


def test_full_size_round_counters(cuda_lib, rmat17):
    """One complete Alg. 2 call at full size (theta = 10^5), every counter compared."""
    q = rmat17
    gh = cuda_lib.load_graph(q.graph)
    got, st = cuda_lib.estimate_decrease(gh, q.seeds, [], q.theta, q.key, 0, stats=True)
    want = oracle_pool.decrease(q.graph, q.seeds, [], q.theta, q.key, 0)
    assert np.array_equal(got, want)
    assert st["samples"] == q.theta


def test_full_size_advanced_greedy_sampled_rounds(cuda_lib, rmat17):
    """AG at full size; rounds 0, 1 and b-1 replayed by the oracle from the GPU's prefix:
    the blocker of round i must be the oracle's argmax given B[:i]."""
    q = rmat17
    gh = cuda_lib.load_graph(q.graph)
    B = cuda_lib.advanced_greedy(gh, q.seeds, q.b, q.theta, q.key)
    assert len(B) == q.b and len(set(B.tolist())) == q.b
    assert not set(B.tolist()) & set(q.seeds.tolist())
    for i in (0, 1, q.b - 1):
        d = oracle_pool.decrease(q.graph, q.seeds, B[:i], q.theta, q.key, i).astype(np.int64)
        d[q.seeds] = -1
        d[B[:i]] = -1
        assert int(np.argmax(d)) == int(B[i]), i


@pytest.mark.parametrize("disable_block_tier", ["0", "1"])
def test_many_seeds(cuda_lib, monkeypatch, disable_block_tier):
    """A seed set too large for the shared-memory warp tier (4,000 seeds): the first tier that
    can hold it takes the samples; counters still match the oracle."""
    rp, col = W.chung_lu(5000, 40000, 2.1, seed=77)
    g = W.Graph(5000, rp, col, W.wc_thresholds(col, 5000))
    seeds = W.uniform_seeds(5000, 4000, seed=78)
    monkeypatch.setenv("IMIN_DISABLE_CTA_TIER", disable_block_tier)
    gh = cuda_lib.load_graph(g)
    got = cuda_lib.estimate_decrease(gh, seeds, [], 500, 4242, 1)
    assert np.array_equal(got, O.decrease(g, seeds, [], 500, 4242, 1))


def test_large_graph_global_bitmap_tier(cuda_lib):
    """n = 2^19 > 2^18: the block tier keeps its visited bitmap in global memory."""
    g = W.graph_rmat_wc(19, 1 << 20, seed=91)
    seeds = W.uniform_seeds(g.n, 30, 92)
    gh = cuda_lib.load_graph(g)
    got, st = cuda_lib.estimate_decrease(gh, seeds, [], 3000, 93, 1, stats=True)
    assert np.array_equal(got, O.decrease(g, seeds, [], 3000, 93, 1))
    assert st["tier_samples"][3] > 0
    B = cuda_lib.advanced_greedy(gh, seeds, 3, 1000, 94)
    assert np.array_equal(B, O.advanced_greedy(g, seeds, 3, 1000, 94))


# --------------------------------------------------------------------------------------------
# large workload: R-MAT 2^22 / 2^26, WC, |S| = 200 (block tier with the bitmap in global memory)
# --------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def rmat22():
    return W.rmat22_query()


def test_rmat22_counters(cuda_lib, rmat22, monkeypatch):
    """At full graph size, 2,000 sampled graphs of round 5 through the default pipeline (block
    tier with the bitmap in global memory) and through the warp-tier pipeline (per-warp global
    hash, then whole-graph scratch), both against the oracle."""
    q = rmat22
    gh = cuda_lib.load_graph(q.graph)
    want = oracle_pool.decrease(q.graph, q.seeds, [], 2000, q.key, 5)
    assert np.array_equal(cuda_lib.estimate_decrease(gh, q.seeds, [], 2000, q.key, 5), want)
    monkeypatch.setenv("IMIN_DISABLE_CTA_TIER", "1")
    assert np.array_equal(cuda_lib.estimate_decrease(gh, q.seeds, [], 2000, q.key, 5), want)


def test_cuda_graph_capture_matches_plain_launches(cuda_lib, tiny, monkeypatch):
    """The greedy rounds run as one captured CUDA graph by default; IMIN_NO_GRAPHS=1 launches them
    one by one. Both must give the same blockers (and the oracle's)."""
    q = tiny
    gh = cuda_lib.load_graph(q.graph)
    g_ag = cuda_lib.advanced_greedy(gh, q.seeds, q.b, 3000, q.key)
    g_gr = cuda_lib.greedy_replace(gh, q.seeds, q.b, 3000, q.key)
    g_bt = cuda_lib.batch_greedy_replace([(gh, q.seeds, q.b, 3000, q.key), (gh, q.seeds[:3], 4, 500, 7)])
    monkeypatch.setenv("IMIN_NO_GRAPHS", "1")
    assert np.array_equal(g_ag, cuda_lib.advanced_greedy(gh, q.seeds, q.b, 3000, q.key))
    assert np.array_equal(g_gr, cuda_lib.greedy_replace(gh, q.seeds, q.b, 3000, q.key))
    p_bt = cuda_lib.batch_greedy_replace([(gh, q.seeds, q.b, 3000, q.key), (gh, q.seeds[:3], 4, 500, 7)])
    assert all(np.array_equal(a, b) for a, b in zip(g_bt, p_bt))
    assert np.array_equal(g_ag, O.advanced_greedy(q.graph, q.seeds, q.b, 3000, q.key))
    # a non-default caller stream
    import torch
    monkeypatch.delenv("IMIN_NO_GRAPHS")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        assert np.array_equal(g_ag, cuda_lib.advanced_greedy(gh, q.seeds, q.b, 3000, q.key))


def test_large_graph_slot_overflow_to_whole_graph_tier(cuda_lib, monkeypatch):
    """n = 2^19 > 2^18 with the block tier's slots capped at 64 local ids: cascades beyond the cap
    are abandoned by the block tier and re-run by the whole-graph tier; counters still equal the
    oracle's. The spread kernel has no fallback and reports the capacity error."""
    g = W.graph_rmat_wc(19, 1 << 20, seed=91)
    seeds = W.uniform_seeds(g.n, 30, 92)
    monkeypatch.setenv("IMIN_CTA_VERTEX_CAP", "64")
    monkeypatch.setenv("IMIN_TIER0_VERTICES", "0")
    gh = cuda_lib.load_graph(g)
    got, st = cuda_lib.estimate_decrease(gh, seeds, [], 1500, 95, 2, stats=True)
    assert np.array_equal(got, O.decrease(g, seeds, [], 1500, 95, 2))
    assert st["tier_samples"][2] > 0 and st["tier_samples"][3] > 0, st
    with pytest.raises(cuda_lib.IminError) as ei:
        cuda_lib.estimate_spread(gh, seeds, [], 1500, 95, 2)
    assert ei.value.code == -4  # IMIN_ERR_CAPACITY
    monkeypatch.delenv("IMIN_CTA_VERTEX_CAP")
    assert cuda_lib.estimate_spread(gh, seeds, [], 1500, 95, 2) == O.spread(g, seeds, [], 1500, 95, 2)


def test_trivalency_rmat_counters_and_greedy_replace(cuda_lib):
    """TR probabilities {0.1, 0.01, 0.001} on an R-MAT 2^13 graph (the single-query path is
    otherwise tested mostly on WC): an Alg. 2 call with a ragged theta, and a full GreedyReplace,
    against the oracle."""
    rp, col = W.rmat(13, 1 << 17, W.RMAT_ABCD, 31)
    g = W.Graph(1 << 13, rp, col, W.tr_thresholds(len(col), 32))
    seeds = W.uniform_seeds(g.n, 25, 33)
    gh = cuda_lib.load_graph(g)
    got = cuda_lib.estimate_decrease(gh, seeds, [7, 11], 2001, 34, 5)
    assert np.array_equal(got, O.decrease(g, seeds, [7, 11], 2001, 34, 5))
    B = cuda_lib.greedy_replace(gh, seeds, 4, 500, 35)
    assert np.array_equal(B, O.greedy_replace(g, seeds, 4, 500, 35))


def test_tuning_is_shared_by_handles_of_one_graph(cuda_lib, monkeypatch):
    """The warp/block cutoff is tuned once per graph and seed-set size class: a second handle of
    the same graph launches only the kernels of its own call (no tuning calls), and both handles
    give the oracle's counters."""
    monkeypatch.delenv("IMIN_TIER0_VERTICES", raising=False)
    monkeypatch.delenv("IMIN_AUTOTUNE", raising=False)
    g = W.graph_rmat_wc(12, 40000, seed=41)
    seeds = W.uniform_seeds(g.n, 20, seed=42)
    want = O.decrease(g, seeds, [], 2000, 43, 1)
    h1 = cuda_lib.load_graph(g)
    c0 = cuda_lib.launch_count()
    assert np.array_equal(cuda_lib.estimate_decrease(h1, seeds, [], 2000, 43, 1), want)
    first = cuda_lib.launch_count() - c0
    h2 = cuda_lib.load_graph(g)
    c0 = cuda_lib.launch_count()
    assert np.array_equal(cuda_lib.estimate_decrease(h2, seeds, [], 2000, 43, 1), want)
    second = cuda_lib.launch_count() - c0
    assert second < first and second <= 6, (first, second)
