"""Python side of O3 (``walks.c``): build with gcc and call through ctypes.

Test infrastructure only (see ``oracle/__init__.py``).  ``build()`` compiles the C
sampler into ``oracle/_build/liboracle_walks.so`` with OpenMP; it shares no
source with the CUDA library.

Pinned by: Philox outputs against Triton's CPU interpreter (an independent
implementation of the same published generator), the expectation of D^(k)
against the exact D(k) of the Power Method and of the rational pair chain
(z-tests), D^ = 1 exactly at din = 0, D = 1-c at din = 1, and thread-count
independence of the counts.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "walks.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_walks.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile walks.c (gcc -O2 -fopenmp) if the shared object is missing or stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.oracle_walk_pairs.restype = ctypes.c_int64
            lib.oracle_walk_pairs.argtypes = [
                ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]
            lib.oracle_philox_many.restype = None
            lib.oracle_philox_many.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
            lib.oracle_walk_threshold.restype = ctypes.c_uint32
            lib.oracle_walk_threshold.argtypes = [ctypes.c_double]
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_walk_pairs_depth.restype = ctypes.c_int64
            lib.oracle_walk_pairs_depth.argtypes = [
                ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]
            lib.oracle_pick_many.restype = None
            lib.oracle_pick_many.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                             ctypes.c_void_p]
            _lib = lib
    return _lib


def philox(counters: np.ndarray, seed: int) -> np.ndarray:
    """Philox-4x32-10 outputs (count, 4) uint32 for counters (count, 4) uint32."""
    ctr = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    _load().oracle_philox_many(ctr.shape[0], ctr.ctypes.data, ctypes.c_uint64(seed), out.ctypes.data)
    return out


def pick(words: np.ndarray, d: int, seed: int = 0) -> np.ndarray:
    """Uniform indices in [0, d) from 32-bit words (rejections redraw from the side stream)."""
    x = np.ascontiguousarray(words, dtype=np.uint32)
    out = np.zeros_like(x)
    _load().oracle_pick_many(x.size, x.ctypes.data, d, ctypes.c_uint64(seed), out.ctypes.data)
    return out


def threshold(c: float) -> int:
    return int(_load().oracle_walk_threshold(c))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def walk_pairs(n: int, in_rowptr, in_col, R, c: float, seed: int, threads: int = 0):
    """(nonmeet uint64[n], pair_steps) for R[k] walk pairs from every node k."""
    rp = np.ascontiguousarray(in_rowptr, dtype=np.int64)
    col = np.ascontiguousarray(in_col, dtype=np.int32)
    R = np.ascontiguousarray(R, dtype=np.uint64)
    if rp.size != n + 1 or R.size != n:
        raise ValueError("shape mismatch")
    nonmeet = np.zeros(n, dtype=np.uint64)
    steps = _load().oracle_walk_pairs(n, rp.ctypes.data, col.ctypes.data, R.ctypes.data,
                                      float(c), ctypes.c_uint64(seed), nonmeet.ctypes.data, int(threads))
    if steps < 0:
        raise ValueError("oracle_walk_pairs rejected its input")
    return nonmeet, int(steps)


def walk_pairs_depth(n: int, in_rowptr, in_col, R, depth, c: float, seed: int, threads: int = 0):
    """(counts uint64[n], pair_steps): nonmeet for depth 0, tail meets (Algorithm 3) for depth > 0."""
    rp = np.ascontiguousarray(in_rowptr, dtype=np.int64)
    col = np.ascontiguousarray(in_col, dtype=np.int32)
    R = np.ascontiguousarray(R, dtype=np.uint64)
    d = np.ascontiguousarray(depth, dtype=np.uint8)
    if rp.size != n + 1 or R.size != n or d.size != n:
        raise ValueError("shape mismatch")
    counts = np.zeros(n, dtype=np.uint64)
    steps = _load().oracle_walk_pairs_depth(n, rp.ctypes.data, col.ctypes.data, R.ctypes.data, d.ctypes.data,
                                            float(c), ctypes.c_uint64(seed), counts.ctypes.data, int(threads))
    if steps < 0:
        raise ValueError("oracle_walk_pairs_depth rejected its input")
    return counts, int(steps)
