"""Python binding of the CUDA C-ABI library (include/imin.h): argument marshalling only.

Every entry point takes the same arguments as its C counterpart. Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA); device work is enqueued on the current torch
CUDA stream unless a stream handle is given. There is no CPU fallback: if libimin.so is not
built or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

IMIN_OK = 0
IMIN_ERR_TIMEOUT = -6
ERRORS = {-1: "invalid argument", -2: "CUDA error", -3: "out of device memory",
          -4: "capacity exceeded", -5: "internal error", -6: "not finished yet"}

_lib = None


class IminError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("samples", ctypes.c_uint64), ("reached", ctypes.c_uint64),
                ("examined_edges", ctypes.c_uint64), ("live_edges", ctypes.c_uint64),
                ("nontree_edges", ctypes.c_uint64), ("dom_passes", ctypes.c_uint64),
                ("tier_samples", ctypes.c_uint64 * 4), ("tier_reached", ctypes.c_uint64 * 4),
                ("tier_examined_edges", ctypes.c_uint64 * 4),
                ("tier_live_edges", ctypes.c_uint64 * 4)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = [int(x) for x in v] if k.startswith("tier_") else int(v)
        return d


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * 6), ("ms", ctypes.c_double * 6)]


class Query(ctypes.Structure):
    """imin_query of include/imin.h."""
    _fields_ = [("graph", ctypes.c_void_p), ("seeds", ctypes.c_void_p), ("n_seeds", ctypes.c_int32),
                ("b", ctypes.c_int32), ("theta", ctypes.c_uint32), ("key", ctypes.c_uint64),
                ("out_blockers", ctypes.c_void_p), ("out_count", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_uint64), ("max_active", ctypes.c_int32),
                ("max_class_samples", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "admitted", "completed", "steps",
                                                "samples", "memory_in_use", "pending")]


KINDS = ("sample_tier0", "sample_tier1", "sample_tier2", "sample_cta", "select", "other")


def lib():
    """Load libimin.so (built by paper_2302_13529_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is not built; run paper_2302_13529_gb300.build.build()")
        L = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        L.imin_load_graph.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P, P, P,
                                      ctypes.POINTER(P)]
        L.imin_load_graph_lt.argtypes = L.imin_load_graph.argtypes
        L.imin_graph_model.argtypes = [P]
        L.imin_free_graph.argtypes = [P]
        L.imin_graph_info.argtypes = [P, P, P]
        L.imin_estimate_decrease.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int32,
                                             ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                             P, P]
        L.imin_estimate_decrease_noalloc.argtypes = L.imin_estimate_decrease.argtypes
        L.imin_estimate_decrease_stats.argtypes = L.imin_estimate_decrease.argtypes[:-1] + [
            ctypes.POINTER(Stats), P]
        for name in ("imin_advanced_greedy", "imin_greedy_replace"):
            getattr(L, name).argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32,
                                         ctypes.c_uint64, P, P, P]
        L.imin_autotune.argtypes = [P, P, ctypes.c_int32, ctypes.c_uint64, P,
                                    ctypes.POINTER(ctypes.c_int32)]
        L.imin_estimate_spread.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_uint32,
                                           ctypes.POINTER(ctypes.c_uint64), P]
        L.imin_estimate_spread_sets.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int32, P, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64,
                                                ctypes.c_uint32, P, P]
        for name in ("imin_baseline_greedy", "imin_exact_blockers"):
            getattr(L, name).argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32,
                                         ctypes.c_uint64, P, P, P]
        L.imin_out_degree_blockers.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, P, P]
        L.imin_random_blockers.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, P, P]
        for name in ("imin_batch_advanced_greedy", "imin_batch_greedy_replace"):
            getattr(L, name).argtypes = [ctypes.POINTER(Query), ctypes.c_int32, P]
        L.imin_autotune_batch.argtypes = [ctypes.POINTER(Query), ctypes.c_int32, ctypes.c_int32, P,
                                          ctypes.POINTER(ctypes.c_int32)]
        L.imin_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]
        L.imin_server_submit.argtypes = [P, ctypes.c_int32, P, P, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_uint32, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_uint64)]
        L.imin_server_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_int64, P, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
        L.imin_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
        L.imin_server_destroy.argtypes = [P]
        L.imin_last_stats.argtypes = [ctypes.POINTER(Stats)]
        L.imin_launch_count.restype = ctypes.c_uint64
        L.imin_profile_enable.argtypes = [ctypes.c_int]
        L.imin_profile_read.argtypes = [ctypes.POINTER(Profile), ctypes.c_int]
        L.imin_last_error.restype = ctypes.c_char_p
        L.imin_abi_version.restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc):
    if rc != IMIN_OK:
        raise IminError(rc, lib().imin_last_error().decode())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(a, dtype):
    """(pointer, keep-alive object, length) for a numpy array or torch tensor."""
    if a is None:
        return None, None, 0
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        want = {np.int32: torch.int32, np.uint32: torch.uint32, np.uint64: torch.uint64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return ctypes.c_void_p(a.data_ptr()), a, a.numel()
    arr = np.ascontiguousarray(np.asarray(a), dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), arr, arr.size


class GraphHandle:
    """A graph resident in device memory (imin_load_graph / imin_load_graph_lt / imin_free_graph).
    model "ic": thr are independent-cascade thresholds; "lt": thr + 1 are the linear-threshold
    shares of each vertex's in-edges."""

    def __init__(self, n, row_ptr, col, thr, stream=None, model="ic"):
        if model not in ("ic", "lt"):
            raise ValueError(f"unknown model {model!r} (ic or lt)")
        rp, k1, _ = _ptr(row_ptr, np.int32)
        c, k2, m = _ptr(col, np.int32)
        t, k3, _ = _ptr(thr, np.uint32)
        h = ctypes.c_void_p()
        load = lib().imin_load_graph if model == "ic" else lib().imin_load_graph_lt
        _check(load(int(n), int(m), rp, c, t, _stream(stream), ctypes.byref(h)))
        self._h = h
        self.n = int(n)
        self.m = int(m)
        self.model = model

    @classmethod
    def from_graph(cls, g, stream=None, model="ic"):
        return cls(g.n, g.row_ptr, g.col, g.thr, stream, model)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            lib().imin_free_graph(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def load_graph(g, stream=None, model="ic") -> GraphHandle:
    return GraphHandle.from_graph(g, stream, model)


def estimate_decrease(gh: GraphHandle, seeds, blocked, theta, key, round_=0, out=None,
                      stream=None, stats=False):
    """imin_estimate_decrease: uint64 counters Delta[n] (numpy unless `out` is given)."""
    s, ks, ns = _ptr(seeds, np.int32)
    b, kb, nb = _ptr(blocked if blocked is not None and len(blocked) else None, np.int32)
    if out is None:
        out = np.zeros(gh.n, dtype=np.uint64)
    o, ko, _ = _ptr(out, np.uint64)
    if stats:
        st = Stats()
        _check(lib().imin_estimate_decrease_stats(gh.handle, s, ns, b, nb, int(theta), int(key),
                                                  int(round_), o, ctypes.byref(st),
                                                  _stream(stream)))
        return out, st.as_dict()
    _check(lib().imin_estimate_decrease(gh.handle, s, ns, b, nb, int(theta), int(key),
                                        int(round_), o, _stream(stream)))
    return out


def estimate_decrease_noalloc(gh: GraphHandle, seeds, blocked, theta, key, round_=0, out=None,
                              stream=None):
    """imin_estimate_decrease_noalloc: the same counters as estimate_decrease, computed without
    allocating memory (working memory comes from the library's static device array)."""
    s, ks, ns = _ptr(seeds, np.int32)
    b, kb, nb = _ptr(blocked if blocked is not None and len(blocked) else None, np.int32)
    if out is None:
        out = np.zeros(gh.n, dtype=np.uint64)
    o, ko, _ = _ptr(out, np.uint64)
    _check(lib().imin_estimate_decrease_noalloc(gh.handle, s, ns, b, nb, int(theta), int(key),
                                                int(round_), o, _stream(stream)))
    return out


def estimate_spread(gh: GraphHandle, seeds, blocked, theta, key, round_=0, stream=None) -> int:
    """imin_estimate_spread: sum over theta sampled graphs of |R| (seeds included); the expected
    spread E(S, G[V \\ B]) is this sum divided by theta."""
    s, ks, ns = _ptr(seeds, np.int32)
    b, kb, nb = _ptr(blocked if blocked is not None and len(blocked) else None, np.int32)
    out = ctypes.c_uint64()
    _check(lib().imin_estimate_spread(gh.handle, s, ns, b, nb, int(theta), int(key), int(round_),
                                      ctypes.byref(out), _stream(stream)))
    return int(out.value)


def autotune(gh: GraphHandle, seeds, key, stream=None) -> int:
    """imin_autotune: re-tune and return the warp/block cutoff for this graph and |seeds|."""
    s, ks, ns = _ptr(seeds, np.int32)
    c = ctypes.c_int32()
    _check(lib().imin_autotune(gh.handle, s, ns, int(key), _stream(stream), ctypes.byref(c)))
    return c.value


def _greedy(fn, gh, seeds, b, theta, key, out, stream):
    s, ks, ns = _ptr(seeds, np.int32)
    if out is None:
        out = np.zeros(max(int(b), 1), dtype=np.int32)
    o, ko, _ = _ptr(out, np.int32)
    cnt = ctypes.c_int32()
    _check(fn(gh.handle, s, ns, int(b), int(theta), int(key), o, ctypes.byref(cnt),
              _stream(stream)))
    return out[:cnt.value]


def advanced_greedy(gh: GraphHandle, seeds, b, theta, key, out=None, stream=None):
    """imin_advanced_greedy (Alg. 3): blockers in selection order."""
    return _greedy(lib().imin_advanced_greedy, gh, seeds, b, theta, key, out, stream)


def greedy_replace(gh: GraphHandle, seeds, b, theta, key, out=None, stream=None):
    """imin_greedy_replace (Alg. 4): blockers in list order."""
    return _greedy(lib().imin_greedy_replace, gh, seeds, b, theta, key, out, stream)


def estimate_spread_sets(gh: GraphHandle, seeds, blocked, sets, theta, key, round_=0, stream=None):
    """imin_estimate_spread_sets: uint64[len(sets)], the simulated spread sum of each blocker set
    (a row of `sets`, blocked on top of `blocked`) over the same theta sampled graphs."""
    s, ks, ns = _ptr(seeds, np.int32)
    b, kb, nb = _ptr(blocked if blocked is not None and len(blocked) else None, np.int32)
    arr = np.ascontiguousarray(np.asarray(sets, dtype=np.int32).reshape(len(sets), -1))
    k = int(arr.shape[1]) if len(sets) else 0
    st, kst, _ = _ptr(arr.reshape(-1) if arr.size else None, np.int32)
    out = np.zeros(max(len(sets), 1), dtype=np.uint64)
    o, ko, _ = _ptr(out, np.uint64)
    _check(lib().imin_estimate_spread_sets(gh.handle, s, ns, b, nb, st, len(sets), k, int(theta), int(key),
                                           int(round_), o, _stream(stream)))
    return out[:len(sets)]


def baseline_greedy(gh: GraphHandle, seeds, b, r, key, out=None, stream=None):
    """imin_baseline_greedy (Alg. 1 with r-sample simulations per candidate)."""
    return _greedy(lib().imin_baseline_greedy, gh, seeds, b, r, key, out, stream)


def exact_blockers(gh: GraphHandle, seeds, b, r, key, out=None, stream=None):
    """imin_exact_blockers: the b-subset of V \\ S with the smallest simulated spread."""
    return _greedy(lib().imin_exact_blockers, gh, seeds, b, r, key, out, stream)


def out_degree_blockers(gh: GraphHandle, seeds, b):
    """imin_out_degree_blockers (OutDegree)."""
    s, ks, ns = _ptr(seeds, np.int32)
    out = np.zeros(max(int(b), 1), dtype=np.int32)
    cnt = ctypes.c_int32()
    _check(lib().imin_out_degree_blockers(gh.handle, s, ns, int(b), out.ctypes.data_as(ctypes.c_void_p),
                                          ctypes.byref(cnt)))
    return out[:cnt.value]


def random_blockers(gh: GraphHandle, seeds, b, key):
    """imin_random_blockers (Rand)."""
    s, ks, ns = _ptr(seeds, np.int32)
    out = np.zeros(max(int(b), 1), dtype=np.int32)
    cnt = ctypes.c_int32()
    _check(lib().imin_random_blockers(gh.handle, s, ns, int(b), int(key), out.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(cnt)))
    return out[:cnt.value]


def _queries(items):
    arr = (Query * max(len(items), 1))()
    keep, outs = [], []
    for i, it in enumerate(items):
        gh, seeds, b, theta, key = it[:5]
        out = it[5] if len(it) > 5 and it[5] is not None else np.zeros(max(int(b), 1), dtype=np.int32)
        s, ks, ns = _ptr(seeds, np.int32)
        o, ko, _ = _ptr(out, np.int32)
        keep += [ks, ko]
        outs.append(out)
        arr[i] = Query(gh.handle.value, s.value if s is not None else None, ns, int(b), int(theta),
                       int(key), o.value, 0)
    return arr, keep, outs


def _batch(fn, items, stream):
    """items: sequence of (GraphHandle, seeds, b, theta, key[, out]) -> list of blocker arrays."""
    arr, keep, outs = _queries(items)
    _check(fn(arr, len(items), _stream(stream)))
    return [outs[i][:arr[i].out_count] for i in range(len(items))]


def autotune_batch(items, driver=0, stream=None) -> int:
    """imin_autotune_batch: pick and cache the queue granularity of this batch; returns it."""
    arr, keep, outs = _queries(items)
    c = ctypes.c_int32()
    _check(lib().imin_autotune_batch(arr, len(items), int(driver), _stream(stream), ctypes.byref(c)))
    return c.value


def batch_advanced_greedy(items, stream=None):
    """imin_batch_advanced_greedy: Alg. 3 for many queries at once (same results as alone)."""
    return _batch(lib().imin_batch_advanced_greedy, items, stream)


def batch_greedy_replace(items, stream=None):
    """imin_batch_greedy_replace: Alg. 4 for many queries at once (same results as alone)."""
    return _batch(lib().imin_batch_greedy_replace, items, stream)


class Server:
    """Continuous-batching request server (imin_server_*): submit queries at any time; each is
    admitted when a batch slot, its device memory and room under its size class's per-step sample
    cap are available, advanced one greedy round per shared step with the other admitted requests
    of its size class (the classes take turns by GPU time), and returns exactly the result of
    running it alone."""

    AG, GR = 0, 1

    def __init__(self, memory_budget: int = 0, max_active: int = 0, max_class_samples: int = 0):
        cfg = ServerConfig(int(memory_budget), int(max_active), int(max_class_samples))
        h = ctypes.c_void_p()
        _check(lib().imin_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, driver, gh: GraphHandle, seeds, b, theta, key) -> int:
        s, ks, ns = _ptr(seeds, np.int32)
        t = ctypes.c_uint64()
        _check(lib().imin_server_submit(self._h, int(driver), gh.handle, s, ns, int(b), int(theta),
                                        int(key), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, capacity: int, timeout_ms: int = -1):
        """(blockers, latency_ms); raises IminError(code=-6) if not finished within timeout_ms."""
        out = np.zeros(max(int(capacity), 1), dtype=np.int32)
        cnt = ctypes.c_int32()
        lat = ctypes.c_double()
        _check(lib().imin_server_wait(self._h, int(ticket), int(timeout_ms),
                                      out.ctypes.data_as(ctypes.c_void_p), int(capacity),
                                      ctypes.byref(cnt), ctypes.byref(lat)))
        return out[:cnt.value], lat.value

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().imin_server_get_stats(self._h, ctypes.byref(st)))
        return {k: int(getattr(st, k)) for k, _ in st._fields_}

    def close(self):
        if self._h is not None and self._h.value:
            lib().imin_server_destroy(self._h)
        self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- measurement hooks ---------------------------------------------------------------------

def last_stats() -> dict:
    """Work counters of the last estimate / greedy call on this thread (imin_last_stats)."""
    st = Stats()
    _check(lib().imin_last_stats(ctypes.byref(st)))
    return st.as_dict()


def launch_count() -> int:
    """Kernels launched by the library so far (imin_launch_count)."""
    return int(lib().imin_launch_count())


def profile_enable(on: bool = True) -> None:
    _check(lib().imin_profile_enable(1 if on else 0))


def profile_read(reset: bool = False) -> dict:
    """Per-kind {launches, ms} accumulated while profiling was enabled (imin_profile_read)."""
    p = Profile()
    _check(lib().imin_profile_read(ctypes.byref(p), 1 if reset else 0))
    return {k: {"launches": int(p.launches[i]), "ms": float(p.ms[i])} for i, k in enumerate(KINDS)}
