"""Seeded synthetic input graphs, shared by the oracle and by the CUDA path.

This module holds no arithmetic of the scheduling method or of BFS, PageRank or colouring.  It
builds int32 CSR graphs shaped like the paper's workloads (Section 6.2, Table 2): RMAT graphs for
the scale-free inputs and 2-D grids with random edge deletion for the mesh-like ones.  All
randomness comes from a counter-based SplitMix64 stream (see ``graphgen.c``), so a (recipe, seed)
pair always gives the same graph on any machine and for any thread count.

The heavy lifting is in ``graphgen.c``; ``build()`` compiles it with gcc into
``libgraphgen.so`` next to this file.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

STREAM_BATCH = 16  # stream id for the sizes of a batched mix
STREAM_ARRIVALS = 17  # stream id for request arrivals and kinds in the serving workload


def build(force: bool = False) -> str:
    """Compiles graphgen.c into libgraphgen.so if it is missing or older than the source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            vp = ctypes.c_void_p
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_uint64, ctypes.c_double, ctypes.c_int, P(vp)]
            lib.gg_grid.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                    P(vp)]
            lib.gg_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, vp, P(vp)]
            lib.gg_destroy.argtypes = [vp]
            lib.gg_num_vertices.argtypes = [vp]
            lib.gg_num_vertices.restype = ctypes.c_int32
            lib.gg_num_entries.argtypes = [vp]
            lib.gg_num_entries.restype = ctypes.c_int64
            lib.gg_copy_out.argtypes = [vp, vp, vp]
            lib.gg_sources.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, vp]
            lib.gg_stream_u64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_relabel.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int, vp, P(vp)]
            lib.gg_stream_u64.restype = ctypes.c_uint64
            _lib = lib
    return _lib


@dataclasses.dataclass
class CSR:
    """A symmetric int32 CSR graph: ``row_ptr`` has n + 1 entries, ``col`` has nnz entries."""

    row_ptr: np.ndarray
    col: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _take(handle: ctypes.c_void_p, name: str) -> CSR:
    lib = _load()
    try:
        n = lib.gg_num_vertices(handle)
        nnz = lib.gg_num_entries(handle)
        rp = np.empty(n + 1, dtype=np.int32)
        col = np.empty(max(nnz, 0), dtype=np.int32)
        rc = lib.gg_copy_out(handle, rp.ctypes.data, col.ctypes.data if nnz else None)
        if rc != 0:
            raise RuntimeError(f"gg_copy_out failed: {rc}")
    finally:
        lib.gg_destroy(handle)
    return CSR(rp, col, name)


def _threads(nthreads):
    return int(nthreads) if nthreads else max(1, min(16, os.cpu_count() or 1))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19, seed: int = 1,
         delete_frac: float = 0.0, nthreads: int | None = None) -> CSR:
    """Undirected RMAT graph: 2**scale vertices, edge_factor * 2**scale sampled edges,
    symmetrised, self-loops and duplicates removed, then ``delete_frac`` of the edges deleted."""
    lib = _load()
    h = ctypes.c_void_p()
    rc = lib.gg_rmat(scale, edge_factor, a, b, c, seed, delete_frac, _threads(nthreads), ctypes.byref(h))
    if rc != 0:
        raise ValueError(f"gg_rmat failed with code {rc}")
    return _take(h, f"rmat{scale}_ef{edge_factor}_s{seed}" + (f"_del{delete_frac:g}" if delete_frac else ""))


def grid(width: int, height: int | None = None, delete_frac: float = 0.0, seed: int = 1,
         nthreads: int | None = None) -> CSR:
    """width x height 4-neighbour grid, vertex id r * width + c, ``delete_frac`` of edges deleted."""
    lib = _load()
    height = width if height is None else height
    h = ctypes.c_void_p()
    rc = lib.gg_grid(width, height, delete_frac, seed, _threads(nthreads), ctypes.byref(h))
    if rc != 0:
        raise ValueError(f"gg_grid failed with code {rc}")
    return _take(h, f"grid{width}x{height}_s{seed}" + (f"_del{delete_frac:g}" if delete_frac else ""))


def from_edges(n: int, pairs, name: str = "edges") -> CSR:
    """Symmetric CSR from undirected pairs (self-loops and duplicates dropped)."""
    lib = _load()
    arr = np.asarray(pairs, dtype=np.int32).reshape(-1, 2)
    eu = np.ascontiguousarray(arr[:, 0])
    ev = np.ascontiguousarray(arr[:, 1])
    h = ctypes.c_void_p()
    rc = lib.gg_from_edges(n, arr.shape[0], eu.ctypes.data if len(eu) else None,
                           ev.ctypes.data if len(ev) else None, ctypes.byref(h))
    if rc != 0:
        raise ValueError(f"gg_from_edges failed with code {rc}")
    return _take(h, name)


def sources(g: CSR, k: int, seed: int = 1) -> np.ndarray:
    """k BFS sources drawn uniformly (with replacement) from the vertices of nonzero degree."""
    lib = _load()
    out = np.empty(k, dtype=np.int32)
    rc = lib.gg_sources(g.row_ptr.ctypes.data, g.n, k, seed, out.ctypes.data)
    if rc != 0:
        raise ValueError(f"gg_sources failed with code {rc}")
    return out


def relabel(g: CSR, seed: int = 1, nthreads: int | None = None):
    """Copy of g with vertex v renamed perm[v] for a seeded uniform random permutation perm, rows
    sorted; returns (copy, perm).  Section 6.4 runs colouring on randomly relabelled ids."""
    lib = _load()
    perm = np.empty(g.n, dtype=np.int32)
    h = ctypes.c_void_p()
    rc = lib.gg_relabel(g.row_ptr.ctypes.data, g.col.ctypes.data if g.nnz else None, g.n, seed, _threads(nthreads),
                        perm.ctypes.data if g.n else None, ctypes.byref(h))
    if rc != 0:
        raise ValueError(f"gg_relabel failed with code {rc}")
    return _take(h, f"{g.name}_relabel{seed}"), perm


def stream_u64(seed: int, stream: int, i: int) -> int:
    return int(_load().gg_stream_u64(seed, stream, i))


def stream_uniform(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """count uniform doubles in [0, 1) from a counter-based stream."""
    return np.array([(stream_u64(seed, stream, start + i) >> 11) * (1.0 / 9007199254740992.0)
                     for i in range(count)], dtype=np.float64)


# ---------------------------------------------------------------------------------------------
# Named workloads (the sizes and recipes of the measured configurations)


def path(n: int) -> CSR:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], f"path{n}")


def cycle(n: int) -> CSR:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"cycle{n}")


def clique(n: int) -> CSR:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"clique{n}")


def star(k: int) -> CSR:
    return from_edges(k + 1, [(0, i) for i in range(1, k + 1)], f"star{k}")


def batched_mix(num_rmat: int = 128, num_grid: int = 128, rmat_scales=(10, 18), grid_sides=(64, 1024),
                delete_frac: float = 0.1, seed: int = 1):
    """The recipe of the batched workload: ``num_rmat`` RMAT graphs (edge factor 16) with scale
    drawn uniformly in ``rmat_scales`` and ``num_grid`` square grids with side drawn uniformly in
    ``grid_sides``, each with ``delete_frac`` of its edges deleted.  Returns a list of
    (kind, size, graph seed) triples; call :func:`materialise` to build one."""
    out = []
    lo, hi = rmat_scales
    for i in range(num_rmat):
        s = lo + int((stream_u64(seed, STREAM_BATCH, 2 * i) >> 11) * (hi - lo + 1) / 9007199254740992.0)
        out.append(("rmat", s, seed * 1000003 + i))
    lo, hi = grid_sides
    for i in range(num_grid):
        w = lo + int((stream_u64(seed, STREAM_BATCH, 2 * i + 1) >> 11) * (hi - lo + 1) / 9007199254740992.0)
        out.append(("grid", w, seed * 1000003 + 500000 + i))
    return out


def materialise(spec, delete_frac: float = 0.1) -> CSR:
    kind, size, gseed = spec
    if kind == "rmat":
        return rmat(size, 16, seed=gseed, delete_frac=delete_frac)
    return grid(size, size, delete_frac=delete_frac, seed=gseed)
