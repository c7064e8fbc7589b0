"""Oracle for the PI batch path: a plain sequential CPU skip list (skiplist.cpp).

TEST INFRASTRUCTURE ONLY. The product path (the CUDA library and its binding) never
imports this package; only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg do. It shares no code with the CUDA path.

``build()`` compiles skiplist.cpp with g++ into ``oracle/_build/liboracle.so``;
``Oracle`` is a thin ctypes wrapper around its C functions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "skiplist.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")

ABSENT, PRESENT, INVALID = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (portable flags only: it builds on x86_64 and aarch64)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        lib.osl_splitmix64.restype = u64
        lib.osl_splitmix64.argtypes = [u64]
        lib.osl_height.restype = i32
        lib.osl_height.argtypes = [u64, i32, u64]
        lib.osl_create.restype = vp
        lib.osl_create.argtypes = [vp, vp, u64, i32, u64, ctypes.POINTER(i32)]
        lib.osl_execute.restype = u64
        lib.osl_execute.argtypes = [vp, vp, vp, vp, u64, vp, vp]
        lib.osl_size.restype = u64
        lib.osl_size.argtypes = [vp]
        lib.osl_export.restype = u64
        lib.osl_export.argtypes = [vp, vp, vp, u64]
        lib.osl_num_levels.restype = i32
        lib.osl_num_levels.argtypes = [vp]
        lib.osl_export_level.restype = u64
        lib.osl_export_level.argtypes = [vp, i32, vp, u64]
        lib.osl_range.restype = u64
        lib.osl_range.argtypes = [vp, vp, vp, u64, vp, vp, vp, u64]
        lib.osl_destroy.restype = None
        lib.osl_destroy.argtypes = [vp]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def splitmix64(x: int) -> int:
    return int(_load().osl_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def height(seed: int, b: int, key: int) -> int:
    return int(_load().osl_height(seed & 0xFFFFFFFFFFFFFFFF, b, key & 0xFFFFFFFFFFFFFFFF))


def promote_exponent(promote_p: float) -> int:
    for b in (1, 2, 3, 4):
        if promote_p == 2.0 ** -b:
            return b
    raise ValueError(f"promote_p must be 1/2, 1/4, 1/8 or 1/16, got {promote_p}")


class Oracle:
    """Sequential skip list: create from (keys, vals), execute batches in arrival order."""

    def __init__(self, keys: np.ndarray, vals: np.ndarray, promote_p: float, seed: int):
        lib = _load()
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        vals = np.ascontiguousarray(vals, dtype=np.uint64)
        err = ctypes.c_int(0)
        self.b = promote_exponent(promote_p)
        self._h = lib.osl_create(_ptr(keys), _ptr(vals), len(keys), self.b,
                                 seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(err))
        if not self._h:
            raise ValueError(f"oracle create failed ({err.value})")

    def execute(self, ops, keys, vals):
        ops = np.ascontiguousarray(ops, dtype=np.uint8)
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        vals = np.ascontiguousarray(vals, dtype=np.uint64)
        n = len(ops)
        rv = np.zeros(n, np.uint64)
        rs = np.zeros(n, np.uint32)
        _load().osl_execute(self._h, _ptr(ops), _ptr(keys), _ptr(vals), n, _ptr(rv), _ptr(rs))
        return rv, rs

    def size(self) -> int:
        return int(_load().osl_size(self._h))

    def export(self):
        n = self.size()
        k = np.zeros(n, np.uint64)
        v = np.zeros(n, np.uint64)
        _load().osl_export(self._h, _ptr(k), _ptr(v), n)
        return k, v

    def range(self, lo, hi):
        """Range search: (offsets[n + 1], keys, vals), query i's pairs in key order at
        [offsets[i], offsets[i + 1])."""
        lib = _load()
        lo = np.ascontiguousarray(lo, dtype=np.uint64)
        hi = np.ascontiguousarray(hi, dtype=np.uint64)
        n = len(lo)
        offs = np.zeros(n + 1, np.uint64)
        total = int(lib.osl_range(self._h, _ptr(lo), _ptr(hi), n, _ptr(offs), None, None, 0))
        k = np.zeros(total, np.uint64)
        v = np.zeros(total, np.uint64)
        lib.osl_range(self._h, _ptr(lo), _ptr(hi), n, _ptr(offs), _ptr(k), _ptr(v), total)
        return offs, k, v

    def num_levels(self) -> int:
        return int(_load().osl_num_levels(self._h))

    def level(self, level: int) -> np.ndarray:
        lib = _load()
        n = int(lib.osl_export_level(self._h, level, None, 0))
        out = np.zeros(n, np.uint64)
        lib.osl_export_level(self._h, level, _ptr(out), n)
        return out

    def close(self):
        if getattr(self, "_h", None):
            _load().osl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
