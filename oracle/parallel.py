"""Multi-threaded (OpenMP) CPU baseline -- MEASUREMENT INFRASTRUCTURE ONLY.

Only ``tests/`` and the CPU-baseline leg of ``bench.py`` may import this module.  It is a timed
comparison program, not the parity reference (that is the serial oracle of this package); the
tests check it against the serial oracle.  Thin ctypes wrappers over ``parallel.c``, which says
what each function computes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "parallel.c")
_LIB = os.path.join(_HERE, "libparallel.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles parallel.c (gcc -fopenmp) into libparallel.so if missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            vp, i32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
            lib.par_bfs.argtypes = [vp, vp, i32, vp, i32, vp, i32]
            lib.par_bfs.restype = ctypes.c_int64
            lib.par_pagerank.argtypes = [vp, vp, i32, f64, f64, i32, vp, i32]
            lib.par_pagerank.restype = i32
            lib.par_color.argtypes = [vp, vp, i32, vp, i32, vp, vp]
            lib.par_color.restype = i32
            _lib = lib
    return _lib


def _csr(g):
    return np.ascontiguousarray(g.row_ptr, dtype=np.int32), np.ascontiguousarray(g.col, dtype=np.int32), int(g.n)


def bfs(g, sources, nthreads: int = 0):
    """Hop distances from each source: (depth [nsrc, n] int32, neighbour entries read)."""
    rp, col, n = _csr(g)
    src = np.ascontiguousarray(sources, dtype=np.int32)
    depth = np.empty((src.size, n), dtype=np.int32)
    e = _load().par_bfs(rp.ctypes.data, col.ctypes.data, n, src.ctypes.data, src.size, depth.ctypes.data, nthreads)
    if e < 0:
        raise ValueError("par_bfs failed")
    return depth, int(e)


def pagerank(g, alpha: float = 0.85, tol_per_vertex: float = 1e-9, max_iter: int = 10000, nthreads: int = 0):
    """Unnormalised fixed point by parallel Jacobi sweeps: (x, sweeps)."""
    rp, col, n = _csr(g)
    x = np.empty(n, dtype=np.float64)
    it = _load().par_pagerank(rp.ctypes.data, col.ctypes.data, n, alpha, tol_per_vertex, max_iter, x.ctypes.data,
                              nthreads)
    if it < 0:
        raise RuntimeError(f"par_pagerank failed ({it})")
    return x, int(it)


def color(g, nthreads: int = 0):
    """Speculative greedy colouring in rounds: (color, count, rounds, neighbour entries read)."""
    rp, col, n = _csr(g)
    c = np.empty(n, dtype=np.int32)
    rounds = ctypes.c_int32(0)
    edges = ctypes.c_int64(0)
    k = _load().par_color(rp.ctypes.data, col.ctypes.data, n, c.ctypes.data, nthreads, ctypes.byref(rounds),
                          ctypes.byref(edges))
    if k < 0:
        raise ValueError("par_color failed")
    return c, int(k), int(rounds.value), int(edges.value)
