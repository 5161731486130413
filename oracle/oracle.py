"""ctypes binding of the C oracle (imin_oracle.c).

TEST INFRASTRUCTURE ONLY: the oracle states what the sampled-dominator-tree estimator
(Alg. 2), the greedy drivers AdvancedGreedy (Alg. 3) and GreedyReplace (Alg. 4), and the
simulated expected spread (Def. 3) compute, slowly and plainly, on the CPU, under the
independent-cascade model (Def. 4) and under the linear-threshold model, the standard triggering
model of Sec. 4.5 (model="lt"). Only the tests, the smoke check and the benchmark's CPU
baseline use it; the product path never imports it.

All functions take numpy arrays; graphs are (n, row_ptr int32[n+1], col int32[m],
thr uint32[m]).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "imin_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libimin_oracle.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile imin_oracle.c into a shared library next to it (plain C, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-pthread", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.oracle_philox4x32_10.restype = None
            L.oracle_edge_word.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_int64]
            L.oracle_edge_word.restype = ctypes.c_uint32
            g = [ctypes.c_int32, ctypes.c_int64, _i32p, _i32p, _u32p]
            L.oracle_sample.argtypes = g + [_i32p, ctypes.c_int32, _i32p, ctypes.c_int32,
                                            ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            _u32p, _i32p, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int64)]
            L.oracle_decrease_range.argtypes = g + [_i32p, ctypes.c_int32, _i32p, ctypes.c_int32,
                                                    ctypes.c_uint64, ctypes.c_uint32,
                                                    ctypes.c_uint32, ctypes.c_uint32, _u64p]
            L.oracle_decrease.argtypes = g + [_i32p, ctypes.c_int32, _i32p, ctypes.c_int32,
                                              ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                              _u64p]
            for name in ("oracle_advanced_greedy", "oracle_greedy_replace"):
                getattr(L, name).argtypes = g + [_i32p, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_uint32, ctypes.c_uint64, _i32p,
                                                 ctypes.POINTER(ctypes.c_int32)]
            L.oracle_spread_range.argtypes = g + [_i32p, ctypes.c_int32, _i32p, ctypes.c_int32,
                                                  ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                                  ctypes.c_uint32, _u64p]
            L.oracle_vertex_word.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_int32]
            L.oracle_vertex_word.restype = ctypes.c_uint32
            L.oracle_set_threads.argtypes = [ctypes.c_int32]
            L.oracle_set_threads.restype = None
            L.oracle_get_threads.restype = ctypes.c_int32
            L.oracle_last_calls.restype = ctypes.c_int32
            L.oracle_spread_sets.argtypes = g + [_i32p, ctypes.c_int32, _i32p, ctypes.c_int32, _i32p,
                                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                                 ctypes.c_uint32, ctypes.c_uint32, _u64p]
            for name in ("oracle_baseline_greedy", "oracle_exact"):
                getattr(L, name).argtypes = g + [_i32p, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_uint32, ctypes.c_uint64, _i32p,
                                                 ctypes.POINTER(ctypes.c_int32)]
            L.oracle_out_degree.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                            _i32p, ctypes.POINTER(ctypes.c_int32)]
            L.oracle_random_blockers.argtypes = [ctypes.c_int32, _i32p, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_uint64, _i32p, ctypes.POINTER(ctypes.c_int32)]
            for name in ("oracle_sample", "oracle_decrease_range", "oracle_decrease",
                         "oracle_advanced_greedy", "oracle_greedy_replace", "oracle_spread_range",
                         "oracle_spread_sets", "oracle_baseline_greedy", "oracle_exact"):
                f = getattr(L, name)
                f.argtypes = f.argtypes + [ctypes.c_int32]  # model: 0 = IC, 1 = LT
                f.restype = ctypes.c_int
            _lib = L
    return _lib


MODELS = {"ic": 0, "lt": 1}


def _model(model: str) -> int:
    if model not in MODELS:
        raise ValueError(f"unknown model {model!r} (ic or lt)")
    return MODELS[model]


def _g(n, row_ptr, col, thr):
    return (int(n), int(len(col)), np.ascontiguousarray(row_ptr, dtype=np.int32),
            np.ascontiguousarray(col, dtype=np.int32), np.ascontiguousarray(thr, dtype=np.uint32))


def _ids(a):
    a = np.ascontiguousarray(np.asarray(a if a is not None else [], dtype=np.int32).reshape(-1))
    if a.size == 0:
        a = np.zeros(1, dtype=np.int32)
        return a, 0
    return a, int(a.size)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its input (rc={rc})")


def set_threads(threads: int) -> None:
    """Worker threads for the sample loops of Alg. 2 and of the spread simulation (default 1,
    the plain sequential loop). The sums over samples are integers, so every thread count gives
    exactly the same results."""
    lib().oracle_set_threads(int(threads))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


class threads:
    """Context manager: run the oracle's sample loops on `count` threads inside the block."""

    def __init__(self, count: int):
        self.count = int(count)

    def __enter__(self):
        self.prev = get_threads()
        set_threads(self.count)
        return self

    def __exit__(self, *exc):
        set_threads(self.prev)


def last_calls() -> int:
    """Alg. 2 calls made by the last advanced_greedy / greedy_replace call of this process
    (GreedyReplace: phase 1 plus the phase-2 calls up to the one that stopped the walk)."""
    return int(lib().oracle_last_calls())


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of a 4-word counter under a 2-word key (SC'11, Sec. 3.3)."""
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(np.asarray(ctr, dtype=np.uint32), np.asarray(key, dtype=np.uint32), out)
    return out


def edge_word(key: int, round_: int, sample: int, e: int) -> int:
    """The uint32 word that decides edge e in sample `sample` of call `round_`."""
    return int(lib().oracle_edge_word(key, round_, sample, e))


def vertex_word(key: int, round_: int, sample: int, v: int) -> int:
    """The uint32 word that decides vertex v's triggering draw in sample `sample` of call
    `round_` (LT model)."""
    return int(lib().oracle_vertex_word(key, round_, sample, v))


def sample(graph, seeds, blocked, key, round_, j, model="ic"):
    """One sampled graph: returns (c[n] subtree sizes, idom[n] global ids or -1, |R|, #live).
    model: "ic" (Def. 4, thr = live threshold) or "lt" (thr + 1 = the edge's share of 2^32)."""
    n, m, rp, col, thr = _g(graph.n, graph.row_ptr, graph.col, graph.thr)
    s, ns = _ids(seeds)
    b, nb = _ids(blocked)
    c = np.zeros(max(n, 1), dtype=np.uint32)
    idom = np.zeros(max(n, 1), dtype=np.int32)
    nr = ctypes.c_int64()
    nl = ctypes.c_int64()
    _check(lib().oracle_sample(n, m, rp, col, thr, s, ns, b, nb, key, round_, j, c, idom,
                               ctypes.byref(nr), ctypes.byref(nl), _model(model)), "sample")
    return c[:n], idom[:n], nr.value, nl.value


def decrease(graph, seeds, blocked, theta, key, round_=0, j0=0, model="ic") -> np.ndarray:
    """Alg. 2 on G[V \\ B]: uint64 Delta[n] = sum of dominator-subtree sizes over samples
    j0 .. j0+theta-1 (no division by theta)."""
    n, m, rp, col, thr = _g(graph.n, graph.row_ptr, graph.col, graph.thr)
    s, ns = _ids(seeds)
    b, nb = _ids(blocked)
    out = np.zeros(max(n, 1), dtype=np.uint64)
    _check(lib().oracle_decrease_range(n, m, rp, col, thr, s, ns, b, nb, key, round_, j0,
                                       j0 + theta, out, _model(model)), "decrease")
    return out[:n]


def spread(graph, seeds, blocked, theta, key, round_=0, j0=0, model="ic") -> int:
    """Def. 3 by simulation: the sum of |R| (seeds included) over samples j0 .. j0+theta-1 of
    call `round_` on G[V \\ B]; the expected-spread estimate is this sum / theta."""
    n, m, rp, col, thr = _g(graph.n, graph.row_ptr, graph.col, graph.thr)
    s, ns = _ids(seeds)
    b, nb = _ids(blocked)
    out = np.zeros(1, dtype=np.uint64)
    _check(lib().oracle_spread_range(n, m, rp, col, thr, s, ns, b, nb, key, round_, j0,
                                     j0 + theta, out, _model(model)), "spread")
    return int(out[0])


def advanced_greedy(graph, seeds, b, theta, key, model="ic") -> np.ndarray:
    """Alg. 3: blockers in selection order."""
    n, m, rp, col, thr = _g(graph.n, graph.row_ptr, graph.col, graph.thr)
    s, ns = _ids(seeds)
    out = np.zeros(max(b, 1), dtype=np.int32)
    cnt = ctypes.c_int32()
    _check(lib().oracle_advanced_greedy(n, m, rp, col, thr, s, ns, b, theta, key, out,
                                        ctypes.byref(cnt), _model(model)), "advanced_greedy")
    return out[:cnt.value].copy()


def greedy_replace(graph, seeds, b, theta, key, model="ic") -> np.ndarray:
    """Alg. 4: blockers in list order (a replacement keeps its predecessor's position)."""
    n, m, rp, col, thr = _g(graph.n, graph.row_ptr, graph.col, graph.thr)
    s, ns = _ids(seeds)
    out = np.zeros(max(b, 1), dtype=np.int32)
    cnt = ctypes.c_int32()
    _check(lib().oracle_greedy_replace(n, m, rp, col, thr, s, ns, b, theta, key, out,
                                       ctypes.byref(cnt), _model(model)), "greedy_replace")
    return out[:cnt.value].copy()


# --------------------------------------------------------------------------------------------
# comparison algorithms of Sec. 5 (evaluated by simulation on the same sampled graphs)
# --------------------------------------------------------------------------------------------

def spread_sets(graph, seeds, blocked, sets, theta, key, round_=0, model="ic") -> np.ndarray:
    """uint64[len(sets)]: for each blocker set (a row of `sets`, added to `blocked`), the sum of
    |R| over samples [0, theta) of call `round_` (common random numbers for all sets)."""
    n, m, rp, col, thr = _g(graph.n, graph.row_ptr, graph.col, graph.thr)
    s, ns = _ids(seeds)
    b, nb = _ids(blocked)
    arr = np.ascontiguousarray(np.asarray(sets, dtype=np.int32).reshape(len(sets), -1))
    k = int(arr.shape[1]) if len(sets) else 0
    flat = arr.reshape(-1) if arr.size else np.zeros(1, np.int32)
    out = np.zeros(max(len(sets), 1), dtype=np.uint64)
    _check(lib().oracle_spread_sets(n, m, rp, col, thr, s, ns, b, nb, flat, len(sets), k, key, round_,
                                    theta, out, _model(model)), "spread_sets")
    return out[:len(sets)]


def baseline_greedy(graph, seeds, b, r, key, model="ic") -> np.ndarray:
    """Alg. 1 BaselineGreedy with r-sample simulations per candidate (round i: samples [0, r) of
    call i for every candidate)."""
    n, m, rp, col, thr = _g(graph.n, graph.row_ptr, graph.col, graph.thr)
    s, ns = _ids(seeds)
    out = np.zeros(max(b, 1), dtype=np.int32)
    cnt = ctypes.c_int32()
    _check(lib().oracle_baseline_greedy(n, m, rp, col, thr, s, ns, b, r, key, out, ctypes.byref(cnt),
                                        _model(model)), "baseline_greedy")
    return out[:cnt.value].copy()


def exact(graph, seeds, b, r, key, model="ic") -> np.ndarray:
    """Exact: the min(b, |V \\ S|)-subset of V \\ S with the smallest simulated spread over samples
    [0, r) of call 0 (the first in lexicographic order among ties), ascending ids."""
    n, m, rp, col, thr = _g(graph.n, graph.row_ptr, graph.col, graph.thr)
    s, ns = _ids(seeds)
    out = np.zeros(max(b, 1), dtype=np.int32)
    cnt = ctypes.c_int32()
    _check(lib().oracle_exact(n, m, rp, col, thr, s, ns, b, r, key, out, ctypes.byref(cnt), _model(model)),
           "exact")
    return out[:cnt.value].copy()


def out_degree_blockers(graph, seeds, b) -> np.ndarray:
    """OutDegree: the b non-seeds of largest out-degree, in that order (smaller id first on ties)."""
    s, ns = _ids(seeds)
    out = np.zeros(max(b, 1), dtype=np.int32)
    cnt = ctypes.c_int32()
    _check(lib().oracle_out_degree(int(graph.n), np.ascontiguousarray(graph.row_ptr, dtype=np.int32), s, ns,
                                   b, out, ctypes.byref(cnt)), "out_degree")
    return out[:cnt.value].copy()


def random_blockers(n, seeds, b, key) -> np.ndarray:
    """Rand: b distinct non-seeds by a Philox-driven partial Fisher-Yates shuffle."""
    s, ns = _ids(seeds)
    out = np.zeros(max(b, 1), dtype=np.int32)
    cnt = ctypes.c_int32()
    _check(lib().oracle_random_blockers(int(n), s, ns, b, key, out, ctypes.byref(cnt)), "random_blockers")
    return out[:cnt.value].copy()
