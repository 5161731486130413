"""Independent checks used to pin the oracle: exact FP64 enumeration of live-edge worlds and
per-sample brute force. Nothing here calls the oracle's BFS, dominator or counter code; the
only shared piece is the per-edge random word (itself pinned by Philox known-answer vectors).
"""
from __future__ import annotations

import itertools
from collections import deque
from fractions import Fraction

import numpy as np

from paper_2302_13529_gb300.workloads import Graph, TWO32

ALWAYS = 0xFFFFFFFF


def edges_of(g: Graph):
    out = []
    for u in range(g.n):
        for e in range(int(g.row_ptr[u]), int(g.row_ptr[u + 1])):
            out.append((e, u, int(g.col[e]), int(g.thr[e])))
    return out


def reach(n, live_edges, seeds, removed=()):
    """Vertices reachable from the seeds over the given (u, v) edges, never entering a vertex
    in `removed` (Def. 2 blockers); seeds are reached at time 0."""
    removed = set(removed)
    adj = [[] for _ in range(n)]
    for u, v in live_edges:
        adj[u].append(v)
    seen = set(s for s in seeds if s not in removed)
    dq = deque(seen)
    while dq:
        u = dq.popleft()
        for v in adj[u]:
            if v not in seen and v not in removed:
                seen.add(v)
                dq.append(v)
    return seen


def exact_moments(g: Graph, seeds, blocked=(), max_uncertain=18):
    """Exact expectation over all live-edge worlds (Def. 4, Lemma 1) in exact rationals for
    edge probabilities (thr+1)/2^32:
      spread          = E[|R|]                       (Def. 3 incl. seeds)
      dec[u]          = E[|R| - |R(g - u)|]          (Thm. 4; = E(S,G) - E(S,G-u))
      dec2[u]         = E[(|R| - |R(g - u)|)^2]      (for the sampling variance)
    Returned as floats."""
    seeds = list(seeds)
    blocked = set(blocked)
    es = edges_of(g)
    certain = [(u, v) for (_, u, v, t) in es if t == ALWAYS]
    unc = [(u, v, Fraction(t + 1, TWO32)) for (_, u, v, t) in es if t != ALWAYS]
    if len(unc) > max_uncertain:
        raise ValueError("too many uncertain edges to enumerate")
    n = g.n
    spread = Fraction(0)
    dec = [Fraction(0)] * n
    dec2 = [Fraction(0)] * n
    for bits in itertools.product((0, 1), repeat=len(unc)):
        pw = Fraction(1)
        live = list(certain)
        for (u, v, p), b in zip(unc, bits):
            if b:
                pw *= p
                live.append((u, v))
            else:
                pw *= 1 - p
        if pw == 0:
            continue
        R = reach(n, live, seeds, blocked)
        spread += pw * len(R)
        for u in R:
            if u in seeds:
                continue
            d = len(R) - len(reach(n, live, seeds, blocked | {u}))
            dec[u] += pw * d
            dec2[u] += pw * d * d
    return float(spread), np.array([float(x) for x in dec]), np.array([float(x) for x in dec2])


def exact_spread_moments(g: Graph, seeds, blocked=(), max_uncertain=18):
    """E[|R|] and E[|R|^2] over all live-edge worlds (Def. 3 incl. seeds), exact rationals for
    edge probabilities (thr+1)/2^32, returned as floats."""
    seeds = list(seeds)
    blocked = set(blocked)
    es = edges_of(g)
    certain = [(u, v) for (_, u, v, t) in es if t == ALWAYS]
    unc = [(u, v, Fraction(t + 1, TWO32)) for (_, u, v, t) in es if t != ALWAYS]
    if len(unc) > max_uncertain:
        raise ValueError("too many uncertain edges to enumerate")
    m1 = Fraction(0)
    m2 = Fraction(0)
    for bits in itertools.product((0, 1), repeat=len(unc)):
        pw = Fraction(1)
        live = list(certain)
        for (u, v, p), b in zip(unc, bits):
            if b:
                pw *= p
                live.append((u, v))
            else:
                pw *= 1 - p
        if pw == 0:
            continue
        r = len(reach(g.n, live, seeds, blocked))
        m1 += pw * r
        m2 += pw * r * r
    return float(m1), float(m2)


def lt_intervals(g: Graph):
    """LT model: the interval [lo, lo + thr] of [0, 2^32) that each edge takes within its
    target's share, in ascending edge id per target."""
    acc = [0] * g.n
    out = {}
    for (e, u, v, t) in edges_of(g):
        out[e] = (acc[v], acc[v] + t)
        acc[v] += t + 1
    assert all(a <= TWO32 for a in acc), "in-edge shares exceed 1"
    return out


def lt_sample_live_edges(g: Graph, key, round_, j, vertex_word):
    """Live edges of LT sample j: edge (u, v) stays iff v's word lies in the edge's interval,
    so every vertex keeps at most one in-edge (its triggering set)."""
    iv = lt_intervals(g)
    words = {}
    live = []
    for (e, u, v, t) in edges_of(g):
        if v not in words:
            words[v] = vertex_word(key, round_, j, v)
        lo, hi = iv[e]
        if lo <= words[v] <= hi:
            live.append((u, v))
    return live


def exact_lt_moments(g: Graph, seeds, blocked=(), max_worlds=1 << 16):
    """Exact expectations over all LT triggering draws (each vertex picks one in-edge with
    probability share/2^32, or none), in exact rationals: (spread, dec[], dec2[]) as in
    exact_moments."""
    seeds = list(seeds)
    blocked = set(blocked)
    choices = {}
    for (e, u, v, t) in edges_of(g):
        choices.setdefault(v, []).append((u, Fraction(t + 1, TWO32)))
    per_vertex = []
    for v, opts in choices.items():
        rest = 1 - sum(p for _, p in opts)
        per_vertex.append([(u, v, p) for u, p in opts] + ([(None, v, rest)] if rest > 0 else []))
    worlds = 1
    for opts in per_vertex:
        worlds *= len(opts)
    if worlds > max_worlds:
        raise ValueError("too many triggering worlds to enumerate")
    n = g.n
    spread = Fraction(0)
    dec = [Fraction(0)] * n
    dec2 = [Fraction(0)] * n
    for pick in itertools.product(*per_vertex):
        pw = Fraction(1)
        live = []
        for (u, v, p) in pick:
            pw *= p
            if u is not None:
                live.append((u, v))
        if pw == 0:
            continue
        R = reach(n, live, seeds, blocked)
        spread += pw * len(R)
        for u in R:
            if u in seeds:
                continue
            d = len(R) - len(reach(n, live, seeds, blocked | {u}))
            dec[u] += pw * d
            dec2[u] += pw * d * d
    return float(spread), np.array([float(x) for x in dec]), np.array([float(x) for x in dec2])


def sample_live_edges(g: Graph, key, round_, j, word):
    """Live edges of sample j: edge e is live iff word(key, round, j, e) <= thr[e] (Def. 4)."""
    return [(u, v) for (e, u, v, t) in edges_of(g) if word(key, round_, j, e) <= t]


def brute_force_sample(g: Graph, seeds, blocked, live):
    """Per-sample truth by vertex deletion (Cor. 1 proof, Thm. 6), on the merged graph where
    edges into seeds are dropped and every seed hangs off the super-seed s':
      u dominates v  <=>  v is not reachable from s' once u is deleted
      c[u]  = |R| - |R(g - u)|                      (= sigma^{->u}, incl. u itself)
      idom(v) = the dominator of v whose own dominator set is largest (the deepest one),
                or -1 when only s' dominates v."""
    n = g.n
    seeds = list(seeds)
    sset = set(seeds)
    blocked = set(blocked)
    live = [(u, v) for (u, v) in live if v not in sset]
    R = reach(n, live, seeds, blocked)
    c = np.zeros(n, dtype=np.int64)
    cut = {}
    for u in R:
        Ru = reach(n, live, seeds, blocked | {u})
        c[u] = len(R) - len(Ru)
        cut[u] = R - Ru
    doms = {v: {u for u in R if u != v and v in cut[u]} for v in R}
    idom = np.full(n, -1, dtype=np.int64)
    for v, ds in doms.items():
        if ds:
            idom[v] = max(ds, key=lambda d: len(doms[d]))
    return R, c, idom
