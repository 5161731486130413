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
