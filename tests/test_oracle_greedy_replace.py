"""Pins for the drivers of the oracle, GreedyReplace (Alg. 4) above all: the order of its list,
the slot a replacement takes, the reverse walk and the early stop of phase 2.

* Two hand-worked graphs with certain edges (tests/golden/greedy_replace_phase2.txt), where
  every counter is an exact integer and the expected lists follow from Alg. 4 by hand. They are
  built so that appending replacements, walking the positions forwards, or dropping the early
  stop each gives a different list.
* Random certain-edge graphs: the drivers restated over brute-force vertex-deletion counts
  (Cor. 1, Thm. 6), which share nothing with the oracle's BFS and dominator code.
* A trace of the oracle's GreedyReplace on the small Chung-Lu workload, replayed call by call
  through the oracle's Alg. 2 with the round numbering of the drivers.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2302_13529_gb300 import workloads as W
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "greedy_replace_phase2.txt")


def load_golden():
    """[(name, graph, seeds, [(alg, b, expected list, Alg. 2 calls)])] from the golden file."""
    out = []
    cur = None
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("["):
            cur = {"name": line.strip("[]"), "want": []}
            out.append(cur)
            continue
        t = line.split()
        if t[0] == "n":
            cur["n"] = int(t[1])
        elif t[0] == "seeds":
            cur["seeds"] = [int(x) for x in t[1].split(",")]
        elif t[0] == "edges":
            cur["edges"] = [tuple(int(x) for x in e.split("-")) for e in t[1:]]
        else:
            cur["want"].append((t[0], int(t[1]), [int(x) for x in t[2].split(",")], int(t[3])))
    res = []
    for c in out:
        g = W.graph_from_edges(c["n"], [(u, v, 1) for u, v in c["edges"]], c["name"])
        res.append((c["name"], g, c["seeds"], c["want"]))
    return res


GOLDEN_CASES = load_golden()


# ------------------------------------------------------------------------------------------
# drivers restated over brute-force counts (certain edges: every sample is G itself)
# ------------------------------------------------------------------------------------------

def _counts(g, seeds, blocked):
    live = [(u, int(v)) for u in range(g.n) for v in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]]
    _, c, _ = pins.brute_force_sample(g, seeds, blocked, live)
    return c


def _best(c, cands):
    """Strict '>' over candidates in ascending id: the smallest id among the maxima."""
    x = -1
    for u in sorted(cands):
        if x == -1 or c[u] > c[x]:
            x = u
    return x


def brute_advanced_greedy(g, seeds, b):
    B = []
    for _ in range(b):
        cands = [u for u in range(g.n) if u not in seeds and u not in B]
        if not cands:
            break
        B.append(_best(_counts(g, seeds, B), cands))
    return B


def brute_greedy_replace(g, seeds, b, variant="faithful"):
    """Alg. 4 with the reading of the golden file; `variant` plants one of the plausible
    mistakes (for the test that shows the pins reject them)."""
    cb = sorted({int(v) for s in seeds for v in g.col[g.row_ptr[s]:g.row_ptr[s + 1]]} - set(seeds))
    B = []
    for _ in range(min(len(cb), b)):
        x = _best(_counts(g, seeds, B), cb)
        cb.remove(x)
        B.append(x)
    k = len(B)
    positions = range(k) if variant == "forward" else range(k - 1, -1, -1)
    for i in positions:
        if variant == "append":
            if i >= len(B):
                continue
            u = B.pop(i)
            rest = list(B)
        else:
            u = B[i]
            rest = B[:i] + B[i + 1:]
        cands = [v for v in range(g.n) if v not in seeds and v not in rest]
        x = _best(_counts(g, seeds, rest), cands)
        if variant == "append":
            B.append(x)
        else:
            B[i] = x
        if x == u and variant != "nobreak":
            break
    return B


# ------------------------------------------------------------------------------------------
# hand-worked graphs
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("case", range(len(GOLDEN_CASES)))
def test_oracle_drivers_match_hand_worked_lists(case):
    name, g, seeds, want = GOLDEN_CASES[case]
    for alg, b, lst, calls in want:
        for key in (1, 77):
            f = O.greedy_replace if alg == "GR" else O.advanced_greedy
            got = [int(x) for x in f(g, seeds, b, 3, key)]
            assert got == lst, (name, alg, b, got, lst)  # exact list equality, order included
            assert O.last_calls() == calls, (name, alg, b, O.last_calls())  # where phase 2 stopped


def test_hand_worked_lists_follow_from_brute_force_counts():
    """The golden lists are what Alg. 4 / Alg. 3 give over exact vertex-deletion counts."""
    for name, g, seeds, want in GOLDEN_CASES:
        for alg, b, lst, _ in want:
            got = brute_greedy_replace(g, seeds, b) if alg == "GR" else brute_advanced_greedy(g, seeds, b)
            assert got == lst, (name, alg, b, got)


@pytest.mark.parametrize("variant", ["append", "forward", "nobreak"])
def test_each_plausible_phase2_mistake_fails_a_golden_list(variant):
    """A replacement appended instead of put in its slot, a forward walk over the positions, or a
    phase 2 without its early stop: each changes at least one hand-worked list."""
    differs = False
    for name, g, seeds, want in GOLDEN_CASES:
        for alg, b, lst, _ in want:
            if alg == "GR" and brute_greedy_replace(g, seeds, b, variant) != lst:
                differs = True
    assert differs, variant


# ------------------------------------------------------------------------------------------
# random certain-edge graphs
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(20))
def test_oracle_drivers_match_brute_force_on_certain_graphs(seed):
    rng = np.random.default_rng(4000 + seed)
    n = int(rng.integers(8, 22))
    g = W.random_small_graph(n, int(rng.integers(n, 3 * n)), seed=4100 + seed, p_choices=(1,))
    k = int(rng.integers(1, 3))
    seeds = [int(x) for x in rng.choice(n, k, replace=False)]
    for b in (1, 2, 4):
        assert [int(x) for x in O.greedy_replace(g, seeds, b, 2, seed)] == brute_greedy_replace(g, seeds, b)
        assert [int(x) for x in O.advanced_greedy(g, seeds, b, 2, seed)] == brute_advanced_greedy(g, seeds, b)


# ------------------------------------------------------------------------------------------
# trace on the small Chung-Lu workload (uncertain edges)
# ------------------------------------------------------------------------------------------

def test_greedy_replace_trace_chung_lu():
    """Alg. 4 call by call: phase-1 call i (round i) picks the best remaining out-neighbour of S
    given the list so far; phase-2 calls (rounds k, k+1, ...) refill positions k-1, k-2, ... with
    the best vertex of V \\ (S u B \\ {u}) and stop at the first x = u. Every call is the oracle's
    Alg. 2 on the prefix; the assembled list must equal the oracle's GreedyReplace exactly."""
    q = W.tiny_chung_lu_query()
    g, seeds, theta, b = q.graph, [int(s) for s in q.seeds], 1500, 6
    sset = set(seeds)
    cb = sorted({int(v) for s in seeds for v in g.col[g.row_ptr[s]:g.row_ptr[s + 1]]} - sset)
    B, rnd = [], 0
    for _ in range(min(b, len(cb))):
        d = O.decrease(g, seeds, B, theta, q.key, rnd).astype(np.int64)
        rnd += 1
        x = max(cb, key=lambda u: (d[u], -u))
        cb.remove(x)
        B.append(x)
    stopped_at = None
    for i in range(len(B) - 1, -1, -1):
        u = B[i]
        rest = B[:i] + B[i + 1:]
        d = O.decrease(g, seeds, rest, theta, q.key, rnd).astype(np.int64)
        rnd += 1
        cands = [v for v in range(g.n) if v not in sset and v not in rest]
        x = max(cands, key=lambda v: (d[v], -v))
        B[i] = x
        if x == u:
            stopped_at = i
            break
    got = [int(x) for x in O.greedy_replace(g, seeds, b, theta, q.key)]
    assert got == B, (got, B, stopped_at)
