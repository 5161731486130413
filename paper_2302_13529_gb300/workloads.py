"""Seeded synthetic inputs: directed power-law graphs, IC edge thresholds, seed sets.

This module only *makes inputs*. It holds none of the estimator's arithmetic and is the one
piece shared by the CUDA path's tests/benchmark and by the CPU oracle's tests: both sides
receive the same arrays from here.

The paper evaluates on SNAP social graphs (Table 4, Sec. 5.1) that are not available offline.
Directed Chung-Lu and R-MAT graphs stand in for them: both give a heavy-tailed degree
distribution like the paper's datasets (average degree 3-60, maximum degree up to ~4% of n).

Edge probabilities follow the two IC models of Sec. 5.1 (Propagation Models):
  * weighted cascade (WC): p(u,v) = 1 / d_in(v)
  * trivalency (TR): p(u,v) drawn uniformly from {0.1, 0.01, 0.001}
Each probability p is stored as a uint32 threshold thr = ceil(p * 2^32) - 1, so that an edge is
live when a uniform uint32 word r satisfies r <= thr; its live probability is (thr + 1) / 2^32,
the smallest multiple of 2^-32 that is >= p. p = 1 maps to 0xFFFFFFFF (always live). Edges with
p = 0 are not stored.
"""
from __future__ import annotations

import ctypes
import dataclasses
import functools
import math
import os
import subprocess
from fractions import Fraction

import numpy as np

TWO32 = 1 << 32


@dataclasses.dataclass
class Graph:
    """Directed graph in CSR form (forward adjacency) with per-edge uint32 thresholds."""

    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col: np.ndarray  # int32[m]
    thr: np.ndarray  # uint32[m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def in_degree(self) -> np.ndarray:
        return np.bincount(self.col, minlength=self.n).astype(np.int64)

    def nbytes(self) -> int:
        return self.row_ptr.nbytes + self.col.nbytes + self.thr.nbytes


# --------------------------------------------------------------------------------------------
# probability -> threshold encoding
# --------------------------------------------------------------------------------------------

def threshold_of(p) -> int:
    """uint32 threshold for probability p in (0, 1]: ceil(p * 2^32) - 1, exact for rationals."""
    f = Fraction(p).limit_denominator(1 << 40) if isinstance(p, float) else Fraction(p)
    if f <= 0 or f > 1:
        raise ValueError("edge probability must lie in (0, 1]")
    num = f.numerator * TWO32
    q = -(-num // f.denominator)  # ceil
    return int(q - 1)


def live_probability(thr) -> np.ndarray:
    """Exact live probability of thresholds (as float64): (thr + 1) / 2^32."""
    return (np.asarray(thr, dtype=np.float64) + 1.0) / float(TWO32)


def wc_thresholds(col: np.ndarray, n: int) -> np.ndarray:
    """Weighted cascade: p(u,v) = 1/d_in(v)  ->  thr = ceil(2^32/d) - 1 = floor((2^32-1)/d)."""
    d_in = np.bincount(col, minlength=n).astype(np.uint64)
    d = d_in[col]
    return ((np.uint64(TWO32 - 1)) // d).astype(np.uint32)


def lt_wc_weights(col: np.ndarray, n: int) -> np.ndarray:
    """Linear-threshold weights b(u,v) = 1/d_in(v), as the shares the LT model takes: edge e into
    v gets floor(2^32/d) of [0, 2^32) (stored as share - 1, the same fixed point as the IC
    thresholds), so that the shares of v's in-edges never exceed 2^32 and each edge keeps
    probability floor(2^32/d)/2^32 <= 1/d."""
    d_in = np.bincount(col, minlength=n).astype(np.uint64)
    d = d_in[col]
    return (np.uint64(TWO32) // d - np.uint64(1)).astype(np.uint32)


TR_PROBS = (Fraction(1, 10), Fraction(1, 100), Fraction(1, 1000))
TR_THRESHOLDS = np.array([threshold_of(p) for p in TR_PROBS], dtype=np.uint32)


def tr_thresholds(m: int, seed: int) -> np.ndarray:
    """Trivalency: each edge independently takes 0.1, 0.01 or 0.001 with probability 1/3."""
    rng = np.random.default_rng(seed)
    return TR_THRESHOLDS[rng.integers(0, 3, size=m)]


# --------------------------------------------------------------------------------------------
# graph generators
# --------------------------------------------------------------------------------------------

def _csr_from_keys(keys: np.ndarray, n: int) -> tuple[np.ndarray, np.ndarray]:
    keys = np.sort(keys)
    src = (keys // n).astype(np.int64)
    dst = (keys % n).astype(np.int32)
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= (1 << 31):
        raise ValueError("graph too large for int32 row offsets")
    return row_ptr.astype(np.int32), dst


def _draw_distinct(draw, n: int, m: int, max_batches: int = 64) -> np.ndarray:
    """Call draw(k) -> (src, dst) until m distinct non-self-loop pairs exist; keep the first m
    distinct pairs in draw order (so the result does not depend on batch boundaries beyond the
    draw sequence itself). Returns int64 keys src*n+dst (unsorted)."""
    pieces = []
    total = 0
    uniq = np.empty(0, dtype=np.int64)
    first = np.empty(0, dtype=np.int64)
    for _ in range(max_batches):
        need = m - len(uniq)
        k = int(max(1024, need * 1.25 + 1024))
        src, dst = draw(k)
        keep = src != dst
        keys = src[keep].astype(np.int64) * n + dst[keep].astype(np.int64)
        pieces.append(keys)
        total += len(keys)
        allk = np.concatenate(pieces)
        uniq, first = np.unique(allk, return_index=True)
        pieces = [allk]
        if len(uniq) >= m:
            order = np.argsort(first, kind="stable")[:m]
            return uniq[order]
    raise RuntimeError("could not draw enough distinct edges; graph too dense for generator")


_GEN_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "graphgen.c")
_GEN_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libimin_gen.so")
_gen = None


def build_generator(force: bool = False) -> str:
    """Compile graphgen.c (plain C) into _build/libimin_gen.so."""
    os.makedirs(os.path.dirname(_GEN_LIB), exist_ok=True)
    if force or not os.path.exists(_GEN_LIB) or os.path.getmtime(_GEN_LIB) < os.path.getmtime(_GEN_SRC):
        tmp = _GEN_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _GEN_SRC, "-lm"])
        os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _genlib():
    global _gen
    if _gen is None:
        L = ctypes.CDLL(build_generator())
        i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        L.imin_gen_chung_lu.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_uint64, i32, i32]
        L.imin_gen_rmat.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, i32, i32]
        _gen = L
    return _gen


def chung_lu(n: int, m: int, gamma: float = 2.1, seed: int = 0, dmax_frac: float = 0.1,
             name: str = "") -> tuple[np.ndarray, np.ndarray]:
    """Directed Chung-Lu graph: expected out- and in-weights w_i = (i + i0)^(-1/(gamma-1)),
    each assigned to vertices by an independent seeded permutation, with i0 chosen so that the
    heaviest vertex expects about dmax_frac * n endpoints; sources drawn with probability
    proportional to w_out and targets proportional to w_in; self-loops and duplicates rejected
    until exactly m distinct edges exist (graphgen.c). Returns (row_ptr, col)."""
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    col = np.zeros(max(m, 1), dtype=np.int32)
    if _genlib().imin_gen_chung_lu(n, m, gamma, dmax_frac, seed & ((1 << 64) - 1), row_ptr, col) != 0:
        raise ValueError("Chung-Lu generation failed (graph too dense?)")
    return row_ptr, col[:m]


RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


def rmat(scale: int, m: int, abcd=RMAT_ABCD, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """R-MAT graph on n = 2^scale vertices: each edge picks one of four quadrants per level
    with probabilities (a, b, c, d); self-loops and duplicates are rejected until exactly m
    distinct edges exist, then vertex ids are relabelled by a seeded random permutation (raw
    R-MAT places the hubs at low ids) (graphgen.c). Returns (row_ptr, col)."""
    a, b, c, d = abcd
    if abs(a + b + c + d - 1.0) > 1e-9:
        raise ValueError("R-MAT quadrant probabilities must sum to 1")
    n = 1 << scale
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    col = np.zeros(max(m, 1), dtype=np.int32)
    if _genlib().imin_gen_rmat(scale, m, a, b, c, seed & ((1 << 64) - 1), row_ptr, col) != 0:
        raise ValueError("R-MAT generation failed")
    return row_ptr, col[:m]


def uniform_seeds(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct seed vertices drawn uniformly without replacement."""
    if k > n:
        raise ValueError("more seeds than vertices")
    rng = np.random.default_rng(seed)
    return rng.choice(n, size=k, replace=False).astype(np.int32)


def query_key(seed: int) -> int:
    """64-bit Philox key for a query, drawn from a seeded generator."""
    rng = np.random.default_rng(seed)
    return int(rng.integers(0, 1 << 63, dtype=np.int64)) * 2 + int(rng.integers(0, 2))


# --------------------------------------------------------------------------------------------
# the five workloads (sizes follow the configurations the method is measured on)
# --------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Query:
    graph: Graph
    seeds: np.ndarray  # int32[k]
    b: int
    theta: int
    key: int


def graph_chung_lu_wc(n, m, seed, name=""):
    rp, col = chung_lu(n, m, 2.1, seed)
    return Graph(n, rp, col, wc_thresholds(col, n), name)


def graph_rmat_wc(scale, m, seed, name=""):
    rp, col = rmat(scale, m, RMAT_ABCD, seed)
    n = 1 << scale
    return Graph(n, rp, col, wc_thresholds(col, n), name)


def tiny_chung_lu_query() -> Query:
    """Chung-Lu n=2,000, m=10,000, WC, |S|=10, b=10, theta=10^4 (the small parity case)."""
    g = graph_chung_lu_wc(2000, 10000, seed=1001, name="chunglu-n2000-m10000-wc")
    return Query(g, uniform_seeds(g.n, 10, 2001), 10, 10_000, query_key(3001))


@functools.lru_cache(maxsize=None)
def _rmat17_graph() -> Graph:
    return graph_rmat_wc(17, 1 << 20, seed=1002, name="rmat17-m2^20-wc")


@functools.lru_cache(maxsize=None)
def _rmat22_graph() -> Graph:
    return graph_rmat_wc(22, 1 << 26, seed=1004, name="rmat22-m2^26-wc")


def rmat17_query(graph: Graph | None = None) -> Query:
    """R-MAT n=2^17, m=2^20, WC, |S|=50, b=50, theta=10^5 (single mid-scale query). The graph is
    generated once per process (its arrays must not be modified)."""
    g = graph or _rmat17_graph()
    return Query(g, uniform_seeds(g.n, 50, 2002), 50, 100_000, query_key(3002))


def batch_queries(count: int = 256, seed: int = 1003) -> list[Query]:
    """256 independent queries on Chung-Lu graphs: n log-uniform in [10^3, 2*10^5], mean degree
    uniform in [5, 20], TR probabilities, |S| uniform in [5, 100], b=20, theta=2*10^4. Generated
    once per process for each (count, seed); the arrays must not be modified."""
    return list(_batch_queries(count, seed))


@functools.lru_cache(maxsize=4)
def _batch_queries(count: int, seed: int) -> tuple:
    out = []
    for q in range(count):
        rng = np.random.default_rng(seed * 1000 + q)
        n = int(math.exp(rng.uniform(math.log(1e3), math.log(2e5))))
        deg = rng.uniform(5.0, 20.0)
        m = int(round(n * deg))
        rp, col = chung_lu(n, m, 2.1, int(rng.integers(1 << 31)))
        thr = tr_thresholds(m, int(rng.integers(1 << 31)))
        g = Graph(n, rp, col, thr, f"chunglu-n{n}-m{m}-tr")
        k = int(rng.integers(5, 101))
        out.append(Query(g, uniform_seeds(n, k, int(rng.integers(1 << 31))), 20, 20_000,
                         query_key(int(rng.integers(1 << 31)))))
    return tuple(out)


def rmat22_query(graph: Graph | None = None) -> Query:
    """R-MAT n=2^22, m=2^26, WC, |S|=200, b=200, theta=2*10^5 (large single query). The graph is
    generated once per process (its arrays must not be modified)."""
    g = graph or _rmat22_graph()
    return Query(g, uniform_seeds(g.n, 200, 2004), 200, 200_000, query_key(3004))


@dataclasses.dataclass
class Request:
    """One serving request: AdvancedGreedy on graph `gi` (0: the R-MAT 2^17 graph, 1: the R-MAT
    2^22 graph) with its own seeds, budget, theta and key."""
    gi: int
    seeds: np.ndarray
    b: int
    theta: int
    key: int


def serving_requests(count: int, seed: int = 5000) -> list[Request]:
    """Requests of the serving workload: each picks the R-MAT 2^17 or the R-MAT 2^22 graph with
    probability 1/2, |S| uniform in [10, 500], b uniform in [10, 100], theta uniform in
    [10^4, 10^5], a seeded 64-bit key."""
    rng = np.random.default_rng(seed)
    ns = (1 << 17, 1 << 22)
    out = []
    for _ in range(count):
        gi = int(rng.integers(0, 2))
        k = int(rng.integers(10, 501))
        seeds = uniform_seeds(ns[gi], k, int(rng.integers(1 << 30)))
        out.append(Request(gi, seeds, int(rng.integers(10, 101)), int(rng.integers(10_000, 100_001)),
                           int(rng.integers(1 << 62))))
    return out


def random_small_graph(n: int, m: int, seed: int, p_choices=None) -> Graph:
    """Uniform random directed graph (no self-loops or duplicate edges) with thresholds drawn
    from p_choices (probabilities); used for small exhaustive and randomized tests."""
    rng = np.random.default_rng(seed)
    m = min(m, n * (n - 1))

    def draw(k):
        return rng.integers(0, n, k), rng.integers(0, n, k)

    keys = _draw_distinct(draw, n, m) if m > 0 else np.empty(0, dtype=np.int64)
    rp, col = _csr_from_keys(keys, n)
    if p_choices is None:
        p_choices = (Fraction(1, 2), Fraction(1, 3), Fraction(9, 10), Fraction(1, 1),
                     Fraction(1, 10))
    thr_choices = np.array([threshold_of(p) for p in p_choices], dtype=np.uint32)
    thr = thr_choices[rng.integers(0, len(thr_choices), size=len(col))]
    return Graph(n, rp, col.astype(np.int32), thr, f"random-n{n}-m{len(col)}")


def graph_from_edges(n: int, edges, name: str = "") -> Graph:
    """CSR graph from a list of (u, v, p) triples (p a probability in (0, 1])."""
    edges = sorted((int(u), int(v), p) for u, v, p in edges)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    for u, _, _ in edges:
        row_ptr[u + 1] += 1
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    col = np.array([v for _, v, _ in edges], dtype=np.int32)
    thr = np.array([threshold_of(p) for _, _, p in edges], dtype=np.uint32)
    return Graph(n, row_ptr, col, thr, name)
