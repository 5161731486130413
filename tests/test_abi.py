"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without a GPU, and
exports every entry point that include/imin.h declares."""
from __future__ import annotations

import ctypes
import os
import re

from paper_2302_13529_gb300 import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "imin.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(imin_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("imin_load_graph", "imin_free_graph", "imin_estimate_decrease",
                 "imin_advanced_greedy", "imin_greedy_replace", "imin_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    lib.imin_abi_version.restype = ctypes.c_int
    assert lib.imin_abi_version() == 1
    lib.imin_last_error.restype = ctypes.c_char_p
    assert lib.imin_last_error() == b""


def test_null_handle_is_rejected_without_gpu_work():
    lib = ctypes.CDLL(build.build())
    assert lib.imin_graph_info(None, None, None) == -1
    assert lib.imin_free_graph(None) == 0


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """The product path has no CPU fallback: with libimin.so missing, the binding raises instead
    of computing anything."""
    import pytest
    from paper_2302_13529_gb300 import imin
    monkeypatch.setattr(imin, "_lib", None)
    monkeypatch.setattr(imin, "LIB", str(tmp_path / "missing" / "libimin.so"))
    with pytest.raises(RuntimeError, match="not built"):
        imin.lib()


def test_invalid_calls_are_rejected_on_the_host():
    """Argument checks that need no GPU work return IMIN_ERR_INVALID with a message."""
    lib = ctypes.CDLL(build.build())
    lib.imin_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    # a malformed CSR: row_ptr does not end at m
    rp = (ctypes.c_int32 * 3)(0, 1, 5)
    col = (ctypes.c_int32 * 1)(0)
    thr = (ctypes.c_uint32 * 1)(1)
    lib.imin_load_graph.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    rc = lib.imin_load_graph(2, 1, ctypes.cast(rp, ctypes.c_void_p), ctypes.cast(col, ctypes.c_void_p),
                             ctypes.cast(thr, ctypes.c_void_p), None, ctypes.byref(out))
    assert rc == -1 and lib.imin_last_error()
    lib.imin_estimate_decrease.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64,
                                            ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.imin_estimate_decrease(None, None, 1, None, 0, 1, 0, 0, None, None) == -1
