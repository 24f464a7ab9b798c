"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gheap.h declares.  CPU only: no compute call is made here.
"""
import ctypes
import os
import re

import pytest

from oracle.genheap import node_of
from paper_1906_06504_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("heap_create", "heap_insert", "heap_delete_min", "heap_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_slot_to_node_is_bit_reversal(lib):
    f = lib.heap_slot_to_node
    f.restype = ctypes.c_uint64
    f.argtypes = [ctypes.c_uint64]
    for j in range(1, 5000):
        assert f(j) == node_of(j)
        assert f(f(j)) == j            # an involution on each level
    assert f(0) == 0


def test_strerror_covers_codes(lib):
    f = lib.heap_strerror
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int]
    texts = {f(c) for c in range(-6, 1)}
    assert len(texts) == 7 and b"unknown error" not in texts
    assert f(-99) == b"unknown error"


def test_create_rejects_bad_arguments(lib):
    # argument checks run before any CUDA call
    f = lib.heap_create
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint64, ctypes.c_uint32,
                  ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]
    h = ctypes.c_void_p()
    assert f(ctypes.byref(h), 1000, 3, 4, 0, 0) == -1      # k not a power of two
    assert f(ctypes.byref(h), 1000, 4096, 4, 0, 0) == -1   # k too large
    assert f(ctypes.byref(h), 1000, 64, 2, 0, 0) == -1     # key_bytes
    assert f(ctypes.byref(h), 0, 64, 4, 0, 0) == -1        # capacity
    assert f(None, 1000, 64, 4, 0, 0) == -1
