"""CPU oracle for BFS, PageRank and greedy colouring -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of ``bench.py`` may
import this package.  The product path (the CUDA library and its Python binding) never loads it,
and the two share no code; they meet only through the seeded graphs of ``graphgen``.

Every function is a thin ctypes wrapper over ``oracle.c``; see that file for what each computes
and which passage of the paper it follows.  ``build()`` compiles it with gcc (single-threaded,
plain C, FP64 for the PageRank arithmetic).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

UNREACHED = 2**31 - 1


def build(force: bool = False) -> str:
    """Compiles oracle.c into liboracle.so if it is missing or older than the source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            lib.oracle_bfs.argtypes = [vp, vp, i32, i32, vp]
            lib.oracle_bfs.restype = i64
            lib.oracle_bfs_certificate.argtypes = [vp, vp, i32, i32, vp, vp]
            lib.oracle_bfs_certificate.restype = ctypes.c_int
            lib.oracle_pagerank.argtypes = [vp, vp, i32, f64, f64, i32, vp, vp, vp]
            lib.oracle_pagerank.restype = ctypes.c_int
            lib.oracle_pr_residual.argtypes = [vp, vp, i32, f64, vp, vp]
            lib.oracle_pr_residual.restype = f64
            lib.oracle_pr_push_serial.argtypes = [vp, vp, i32, f64, f64, vp, vp, vp]
            lib.oracle_pr_push_serial.restype = i64
            lib.oracle_greedy_color.argtypes = [vp, vp, i32, vp, vp]
            lib.oracle_greedy_color.restype = i32
            lib.oracle_check_coloring.argtypes = [vp, vp, i32, vp, vp, vp]
            lib.oracle_check_coloring.restype = ctypes.c_int
            _lib = lib
    return _lib


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    return rp, col, rp.shape[0] - 1


def _p(a):
    return a.ctypes.data if a is not None and a.size else None


def bfs(g, src: int) -> np.ndarray:
    """Hop distances from src (int32; UNREACHED = INT32_MAX outside src's component)."""
    rp, col, n = _csr(g)
    depth = np.empty(n, dtype=np.int32)
    r = _load().oracle_bfs(_p(rp), _p(col), n, int(src), _p(depth))
    if r < 0:
        raise ValueError("oracle_bfs: bad arguments")
    return depth


def bfs_certificate(g, src: int, depth) -> tuple[int, int]:
    """(code, vertex): code 0 if depth[] is the hop-distance vector from src, else the failed
    property (1 source, 2 closure, 3 edge difference, 4 parent) and the offending vertex."""
    rp, col, n = _csr(g)
    d = np.ascontiguousarray(depth, dtype=np.int32)
    bad = ctypes.c_int32(-1)
    code = _load().oracle_bfs_certificate(_p(rp), _p(col), n, int(src), _p(d), ctypes.byref(bad))
    return int(code), int(bad.value)


def pagerank(g, alpha: float = 0.85, tol_per_vertex: float = 1e-13, max_iter: int = 10000):
    """FP64 fixed point of x = (1 - alpha) 1 + alpha P x (unnormalised; sum ~ n).
    Returns (x, sweeps, last_step_l1)."""
    rp, col, n = _csr(g)
    x = np.empty(n, dtype=np.float64)
    it = ctypes.c_int32(0)
    delta = ctypes.c_double(0)
    rc = _load().oracle_pagerank(_p(rp), _p(col), n, float(alpha), float(tol_per_vertex), int(max_iter), _p(x),
                                 ctypes.byref(it), ctypes.byref(delta))
    if rc < 0:
        raise ValueError("oracle_pagerank: bad arguments")
    if rc == 1:
        raise RuntimeError(f"oracle_pagerank did not converge in {max_iter} sweeps (last step {delta.value})")
    return x, int(it.value), float(delta.value)


def pagerank_sweeps(g, alpha: float, sweeps: int) -> np.ndarray:
    """Exactly ``sweeps`` power-iteration sweeps from x = 1 (for bounded timing samples)."""
    rp, col, n = _csr(g)
    x = np.empty(n, dtype=np.float64)
    it = ctypes.c_int32(0)
    delta = ctypes.c_double(0)
    _load().oracle_pagerank(_p(rp), _p(col), n, float(alpha), 0.0, int(sweeps), _p(x), ctypes.byref(it),
                            ctypes.byref(delta))
    return x


def pr_residual(g, x, alpha: float = 0.85):
    """(rho, ||rho||_1) for rho = (1 - alpha) 1 + alpha P x - x, in FP64; x unnormalised."""
    rp, col, n = _csr(g)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    rho = np.empty(n, dtype=np.float64)
    l1 = _load().oracle_pr_residual(_p(rp), _p(col), n, float(alpha), _p(xx), _p(rho))
    return rho, float(l1)


def fixed_point_sum(g, alpha: float = 0.85) -> float:
    """Exact sum of the unnormalised fixed point: n - alpha * (number of isolated vertices).

    1^T (I - alpha P) = (1 - alpha) 1^T on columns of nonzero degree, so each connected part
    sums to its vertex count, and an isolated vertex keeps 1 - alpha."""
    deg = np.diff(np.asarray(g.row_ptr, dtype=np.int64))
    return float(deg.shape[0] - alpha * np.count_nonzero(deg == 0))


def pr_error_bound(g, q, alpha: float = 0.85) -> float:
    """A posteriori bound on ||q - p/sum(p)||_1 for a normalised candidate q (sum 1), from the
    FP64 residual: with x = q sum(p), ||x - p||_1 <= ||rho(x)||_1 / (1 - alpha), because the
    inverse of (I - alpha P) has induced L1 norm at most 1 / (1 - alpha)."""
    q = np.asarray(q, dtype=np.float64)
    s = fixed_point_sum(g, alpha)
    _, l1 = pr_residual(g, q * s, alpha)
    return l1 / ((1.0 - alpha) * s)


def pr_push_serial(g, alpha: float = 0.85, eps: float = 1e-9):
    """Serial push-residual PageRank (Algorithm 3's steps, FIFO order).
    Returns (rank, residue, pushes, edge_pushes), FP64, unnormalised."""
    rp, col, n = _csr(g)
    rank = np.empty(n, dtype=np.float64)
    res = np.empty(n, dtype=np.float64)
    ep = ctypes.c_int64(0)
    pushes = _load().oracle_pr_push_serial(_p(rp), _p(col), n, float(alpha), float(eps), _p(rank), _p(res),
                                           ctypes.byref(ep))
    if pushes < 0:
        raise ValueError("oracle_pr_push_serial: bad arguments")
    return rank, res, int(pushes), int(ep.value)


def greedy_color(g, order=None) -> tuple[np.ndarray, int]:
    """Serial first-fit colouring in ``order`` (default: vertex id order). Returns (color, count)."""
    rp, col, n = _csr(g)
    color = np.empty(n, dtype=np.int32)
    o = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    k = _load().oracle_greedy_color(_p(rp), _p(col), n, _p(o), _p(color))
    if k < 0:
        raise ValueError("oracle_greedy_color: bad arguments")
    return color, int(k)


def check_coloring(g, color) -> tuple[int, int, int]:
    """(code, vertex, num_colors): code 0 if proper with 0 <= c(v) <= deg(v); 1 conflict,
    2 out of range, 3 uncoloured."""
    rp, col, n = _csr(g)
    c = np.ascontiguousarray(color, dtype=np.int32)
    bad = ctypes.c_int32(-1)
    k = ctypes.c_int32(0)
    code = _load().oracle_check_coloring(_p(rp), _p(col), n, _p(c), ctypes.byref(bad), ctypes.byref(k))
    return int(code), int(bad.value), int(k.value)
