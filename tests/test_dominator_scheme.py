"""The dominator scheme of the GPU kernels, restated in plain Python and checked against
networkx (CPU). The kernels number the reached vertices in BFS discovery order, start every
idom(v) at v's BFS parent and fold idom(v) <- NCA(idom(v), p, parent(v)) over the non-tree
in-edges (p -> v) until a pass changes nothing. The ancestor chains start as BFS-tree paths,
supersets of the dominator sets, and every fold keeps them supersets; at the fixed point every
in-edge has idom(v) above its source, so they are the dominator sets (Defs. 5-6). This test pins
that scheme, independently of the CUDA code, on
random graphs: in sequential order, in shuffled order, and with every pass reading a snapshot
taken at its start (the most stale view concurrent threads can have); and it shows why the
parent edge must be folded too."""
from __future__ import annotations

import random
from collections import deque

import networkx as nx
import pytest


def bfs_numbering(n, adj, seeds):
    """Local ids: 0 = super-seed, seeds 1..|S|, then BFS discovery order; parent[] and the
    non-tree edges (p, v) between reached vertices, edges into seeds dropped."""
    lid = {s: i + 1 for i, s in enumerate(seeds)}
    order = [None] + list(seeds)
    parent = [0] * (len(seeds) + 1)
    edges = []
    front = list(seeds)
    while front:
        nxt = []
        for u in front:
            for v in adj[u]:
                if v in seeds:
                    continue
                if v not in lid:
                    lid[v] = len(order)
                    order.append(v)
                    parent.append(lid[u])
                    nxt.append(v)
                elif lid[v] != lid[u]:
                    edges.append((lid[u], lid[v]))
        front = nxt
    return order, parent, edges


def nca(idom, a, b):
    while a != b:
        if a > b:
            a = idom[a]
        else:
            b = idom[b]
    return a


def fold(parent, edges, mode, with_parent, rng):
    idom = list(parent)
    for _ in range(len(parent) + 2):
        snap = list(idom) if mode == "snapshot" else idom
        es = list(edges)
        if mode == "shuffled":
            rng.shuffle(es)
        changed = False
        for p, v in es:
            a = nca(snap, snap[v], p)
            if with_parent:
                a = nca(snap, a, parent[v])
            if a < idom[v]:
                idom[v] = a
                changed = True
        if not changed:
            return idom
    raise AssertionError("no fixed point")


def truth(order, adj, seeds):
    """Immediate dominators from networkx on the merged graph (root -> every seed)."""
    G = nx.DiGraph()
    root = "root"
    reached = set(order[1:])
    for s in seeds:
        G.add_edge(root, s)
    for u in reached:
        for v in adj[u]:
            if v in reached and v not in seeds:
                G.add_edge(u, v)
    return nx.immediate_dominators(G, root)


def random_case(seed):
    rng = random.Random(seed)
    n = rng.randint(4, 30)
    m = rng.randint(n, 4 * n)
    adj = [[] for _ in range(n)]
    for _ in range(m):
        u, v = rng.randrange(n), rng.randrange(n)
        if u != v and v not in adj[u]:
            adj[u].append(v)
    seeds = rng.sample(range(n), rng.randint(1, 3))
    return n, adj, seeds


@pytest.mark.parametrize("mode", ["sequential", "shuffled", "snapshot"])
def test_bfs_order_nca_folding_gives_the_dominator_tree(mode):
    rng = random.Random(7)
    for seed in range(1500):
        n, adj, seeds = random_case(seed)
        order, parent, edges = bfs_numbering(n, adj, seeds)
        idom = fold(parent, edges, mode, True, rng)
        want = truth(order, adj, seeds)
        for i in range(len(seeds) + 1, len(order)):
            got = "root" if idom[i] == 0 else order[idom[i]]
            assert got == want[order[i]], (seed, mode, order[i])


def test_folding_without_the_parent_edge_can_stop_too_deep():
    """Folding only the non-tree edges can leave idom(v) below the true dominator when the
    parent's own chain moves up later; the kernels fold the parent edge in every pass."""
    rng = random.Random(3)
    bad = 0
    for seed in range(3000):
        n, adj, seeds = random_case(seed)
        order, parent, edges = bfs_numbering(n, adj, seeds)
        idom = fold(parent, edges, "shuffled", False, rng)
        want = truth(order, adj, seeds)
        bad += any(("root" if idom[i] == 0 else order[idom[i]]) != want[order[i]]
                   for i in range(len(seeds) + 1, len(order)))
    assert bad > 0
