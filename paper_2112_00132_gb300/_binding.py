"""ctypes binding of the C ABI declared in include/atos.h (argument marshalling only).

Every step of BFS, PageRank and colouring runs in the CUDA kernels of ``libatos.so``; this module
only converts Python / torch arguments into the plain pointers and sizes of the C entry points.
PyTorch provides device memory (output tensors) and streams.  There is no CPU fallback: if the
library is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libatos.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "atos.h")

# status codes and constants (mirrors include/atos.h)
OK = 0
ERR_INVALID_ARG = -1
ERR_BAD_CSR = -2
ERR_OOM = -3
ERR_QUEUE_OVERFLOW = -4
ERR_TIMEOUT = -5
ERR_CUDA = -6
ERR_UNSUPPORTED = -7
ERR_BUSY = -8
ERR_BOUNDS = -9

WORKER_WARP = 32
WORKER_THREAD = 1
PERSISTENT, DISCRETE, BSP = 0, 1, 2
FETCH_FIXED, FETCH_GREEDY, FETCH_SPREAD = 0, 1, 2
FLAG_PHANTOM_TASK = 1
FLAG_PR_CROSSING = 2
FLAG_SPREAD_IDS = 4
FLAG_USE_TUNED = 8
FLAG_GC_ORDERED = 16
FLAG_BFS_EXPAND_ONCE = 32
FLAG_BSP_DEVICE_LOOP = 64
FLAG_BSP_PER_SOURCE = 128
FLAG_GC_DEPENDENCY = 256
FLAG_BFS_SPLIT_ROWS = 512
DEVICE_PTRS, BORROW, CHECK_SYMMETRIC, SKIP_VALIDATION = 1, 2, 4, 8
UNREACHED = 2**31 - 1


class Config(ctypes.Structure):
    _fields_ = [
        ("worker_size", ctypes.c_int32),
        ("fetch_size", ctypes.c_int32),
        ("strategy", ctypes.c_int32),
        ("fetch_policy", ctypes.c_int32),
        ("num_blocks", ctypes.c_int32),
        ("check_size", ctypes.c_int32),
        ("window", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("queue_capacity", ctypes.c_int64),
        ("spin_limit_ns", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

    def __repr__(self):
        return f"Config({self.as_dict()})"


class Stats(ctypes.Structure):
    _fields_ = [
        ("ms", ctypes.c_double),
        ("tasks", ctypes.c_int64),
        ("edges", ctypes.c_int64),
        ("pushes", ctypes.c_int64),
        ("iterations", ctypes.c_int64),
        ("residual_l1", ctypes.c_double),
        ("error_bound", ctypes.c_double),
        ("num_colors", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("batches", ctypes.c_int64),
        ("idle_polls", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


APP_BFS, APP_PAGERANK, APP_COLOR = 0, 1, 2


class Instance(ctypes.Structure):
    _fields_ = [
        ("app", ctypes.c_int32),
        ("graph", ctypes.c_int32),
        ("source", ctypes.c_int32),
        ("alpha", ctypes.c_float),
        ("eps", ctypes.c_float),
        ("reserved", ctypes.c_int32),
        ("out", ctypes.c_void_p),
    ]


class Completion(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_int64),
        ("status", ctypes.c_int32),
        ("app", ctypes.c_int32),
        ("graph", ctypes.c_int32),
        ("num_colors", ctypes.c_int32),
        ("tasks", ctypes.c_int64),
        ("edges", ctypes.c_int64),
        ("epochs", ctypes.c_int64),
        ("error_bound", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AtosError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})" if what else status_string(status))


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libatos.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u32, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_float
        P = ctypes.POINTER
        L.atos_queue_config.argtypes = [P(Config), ctypes.c_char_p]
        L.atos_csr_validate.argtypes = [vp, vp, i32, i64, u32]
        L.atos_graph_create.argtypes = [vp, vp, i32, i64, u32, vp, P(vp)]
        L.atos_graph_destroy.argtypes = [vp]
        L.atos_graph_info.argtypes = [vp, P(i32), P(i64), P(i32)]
        L.atos_bfs.argtypes = [vp, vp, i32, vp, P(Config), vp, P(Stats)]
        L.atos_pagerank.argtypes = [vp, f32, f32, vp, P(Config), vp, P(Stats)]
        L.atos_color.argtypes = [vp, vp, P(i32), P(Config), vp, P(Stats)]
        L.atos_debug_queue_state.argtypes = [vp, i32, vp, vp, P(i32)]
        L.atos_debug_queue_state.restype = ctypes.c_int
        L.atos_batch_create.argtypes = [vp, i32, P(Instance), i32, P(Config), P(vp)]
        L.atos_batch_run.argtypes = [vp, vp]
        L.atos_batch_run_graph.argtypes = [vp, vp]
        L.atos_batch_stats.argtypes = [vp, P(Stats), P(Stats), vp]
        L.atos_batch_info.argtypes = [vp, P(i32), P(i32), P(i32)]
        L.atos_batch_destroy.argtypes = [vp]
        for name in ("atos_batch_create", "atos_batch_run", "atos_batch_run_graph", "atos_batch_stats",
                     "atos_batch_info", "atos_batch_destroy"):
            getattr(L, name).restype = ctypes.c_int
        L.atos_server_create.argtypes = [vp, i32, i32, i64, P(Config), P(vp)]
        L.atos_server_submit.argtypes = [vp, P(Instance), P(i64)]
        L.atos_server_step.argtypes = [vp, i64, P(i32)]
        L.atos_server_poll.argtypes = [vp, P(Completion), i32, P(i32)]
        L.atos_server_info.argtypes = [vp, P(i32), P(i64), P(i64), P(i64)]
        L.atos_server_destroy.argtypes = [vp]
        for name in ("atos_server_create", "atos_server_submit", "atos_server_step", "atos_server_poll",
                     "atos_server_info", "atos_server_destroy"):
            getattr(L, name).restype = ctypes.c_int
        L.atos_timeline.argtypes = [vp, i64, i32]
        L.atos_timeline.restype = ctypes.c_int
        L.atos_timeline_read.argtypes = [vp, vp, vp, i32]
        L.atos_timeline_read.restype = ctypes.c_int
        L.atos_pool_trim.argtypes = [P(i64)]
        L.atos_pool_trim.restype = ctypes.c_int
        L.atos_edge_ceiling.argtypes = [vp, i32, i32, P(ctypes.c_double), vp]
        L.atos_edge_ceiling.restype = ctypes.c_int
        L.atos_autotune.argtypes = [vp, i32, vp, i32, vp, i32, P(Config), P(ctypes.c_double), vp]
        L.atos_autotune.restype = ctypes.c_int
        L.atos_batch_autotune.argtypes = [vp, i32, P(Instance), i32, i32, P(Config), P(ctypes.c_double), vp]
        L.atos_batch_autotune.restype = ctypes.c_int
        L.atos_tuned_config.argtypes = [vp, i32, P(Config)]
        L.atos_tuned_config.restype = ctypes.c_int
        L.atos_bfs_noalloc.argtypes = [vp, vp, i32, i64, i32, vp, vp]
        L.atos_bfs_noalloc.restype = ctypes.c_int
        L.atos_debug_spread_layout.argtypes = [vp, vp, P(i32), vp]
        L.atos_debug_spread_layout.restype = ctypes.c_int
        L.atos_debug_scratch_check.argtypes = [vp, P(ctypes.c_uint64), P(ctypes.c_uint64)]
        L.atos_debug_scratch_check.restype = ctypes.c_int
        L.atos_kernel_launches.argtypes = []
        L.atos_kernel_launches.restype = ctypes.c_uint64
        L.atos_status_string.argtypes = [ctypes.c_int]
        L.atos_status_string.restype = ctypes.c_char_p
        L.atos_version.restype = ctypes.c_char_p
        for name in ("atos_queue_config", "atos_csr_validate", "atos_graph_create", "atos_graph_destroy",
                     "atos_graph_info", "atos_bfs", "atos_pagerank", "atos_color"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the functions declared in an include/*.h header."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(atos_\w+)\s*\(", text)) - {"atos_graph_t"})


def kernel_launches() -> int:
    """Kernels the library has launched so far in this process."""
    return int(lib().atos_kernel_launches())


def status_string(status: int) -> str:
    return lib().atos_status_string(int(status)).decode()


def version() -> str:
    return lib().atos_version().decode()


def queue_config(preset: str | None = None, **overrides) -> Config:
    """A config filled from a preset ("default", "persist-warp", "persist-cta", "discrete-cta",
    "discrete-warp", "bsp"), then with the given fields overridden."""
    cfg = Config()
    rc = lib().atos_queue_config(ctypes.byref(cfg), preset.encode() if preset else None)
    if rc != OK:
        raise AtosError(rc, f"atos_queue_config({preset!r})")
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise AttributeError(k)
        setattr(cfg, k, v)
    return cfg


def csr_validate(row_ptr, col, check_symmetric: bool = False) -> int:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    c = np.ascontiguousarray(col, dtype=np.int32)
    return int(lib().atos_csr_validate(rp.ctypes.data, c.ctypes.data if c.size else None, rp.shape[0] - 1,
                                       c.shape[0], CHECK_SYMMETRIC if check_symmetric else 0))


def _stream_handle(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc: int, what: str):
    if rc != OK:
        raise AtosError(rc, what)


class Graph:
    """An undirected int32 CSR graph resident on the GPU (wraps an atos_graph_t).

    ``row_ptr`` / ``col`` may be numpy arrays (host; validated on the host and copied) or torch
    CUDA int32 tensors (device; ``borrow=True`` uses them in place)."""

    def __init__(self, row_ptr, col, *, borrow: bool = False, check_symmetric: bool = False,
                 skip_validation: bool = False, stream=None):
        self._h = ctypes.c_void_p()
        self._keep = None
        flags = (CHECK_SYMMETRIC if check_symmetric else 0) | (SKIP_VALIDATION if skip_validation else 0)
        if hasattr(row_ptr, "is_cuda") and row_ptr.is_cuda:
            import torch
            assert row_ptr.dtype == torch.int32 and col.dtype == torch.int32
            rp, c = row_ptr.contiguous(), col.contiguous()
            flags |= DEVICE_PTRS | (BORROW if borrow else 0)
            if borrow:
                self._keep = (rp, c)
            n, nnz = rp.numel() - 1, c.numel()
            rc = lib().atos_graph_create(rp.data_ptr(), c.data_ptr() if nnz else None, n, nnz, flags,
                                         _stream_handle(stream), ctypes.byref(self._h))
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
            c = np.ascontiguousarray(col, dtype=np.int32)
            n, nnz = rp.shape[0] - 1, c.shape[0]
            rc = lib().atos_graph_create(rp.ctypes.data, c.ctypes.data if nnz else None, n, nnz, flags,
                                         _stream_handle(stream), ctypes.byref(self._h))
        _check(rc, "atos_graph_create")
        n_, nnz_, md = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
        _check(lib().atos_graph_info(self._h, ctypes.byref(n_), ctypes.byref(nnz_), ctypes.byref(md)),
               "atos_graph_info")
        self.n, self.nnz, self.max_degree = n_.value, nnz_.value, md.value

    @classmethod
    def from_csr(cls, g, **kw):
        """From any object with ``row_ptr`` and ``col`` arrays (e.g. graphgen.CSR)."""
        return cls(g.row_ptr, g.col, **kw)

    def close(self):
        if self._h:
            lib().atos_graph_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def queue_state(self, ninst: int):
        """(tail, completed, head) per instance of the last launch, and the failed wait site."""
        words = np.zeros(ninst, dtype=np.uint64)
        heads = np.zeros(ninst, dtype=np.uint32)
        site = ctypes.c_int32(0)
        _check(lib().atos_debug_queue_state(self._h, ninst, words.ctypes.data, heads.ctypes.data,
                                            ctypes.byref(site)), "atos_debug_queue_state")
        return [(int(w >> 32), int(w & 0xffffffff), int(h)) for w, h in zip(words, heads)], site.value

    def spread_layout(self, stream=None):
        """(perm, hubs) of the spread-id copy: perm[v] is the copy's id of v, ids [0, hubs) the hub
        region."""
        n = ctypes.c_int32()
        lib().atos_graph_info(self._h, ctypes.byref(n), None, None)
        perm = np.zeros(max(n.value, 1), dtype=np.int32)
        hubs = ctypes.c_int32(0)
        _check(lib().atos_debug_spread_layout(self._h, perm.ctypes.data, ctypes.byref(hubs), _stream_handle(stream)),
               "atos_debug_spread_layout")
        return perm[:n.value], hubs.value

    def scratch_check(self):
        """(set queued bits, occupied ring slots) after the last run; both 0 after a clean run."""
        bits, slots = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().atos_debug_scratch_check(self._h, ctypes.byref(bits), ctypes.byref(slots)),
               "atos_debug_scratch_check")
        return bits.value, slots.value

    def autotune(self, app: str, sources=None, repeats: int = 2, stream=None):
        """Times the candidate configurations of ``app`` ("bfs", "pagerank", "color") on this
        graph; returns (best Config, its device ms) and caches it for the graph's class."""
        import torch
        code = {"bfs": APP_BFS, "pagerank": APP_PAGERANK, "color": APP_COLOR}[app]
        src = np.ascontiguousarray(np.atleast_1d(np.asarray(sources if sources is not None else [0])),
                                   dtype=np.int32)
        rows = src.shape[0] if code == APP_BFS else 1
        scratch = torch.empty((rows, max(self.n, 1)), dtype=torch.int32, device="cuda")
        best, ms = Config(), ctypes.c_double(0)
        _check(lib().atos_autotune(self._h, code, src.ctypes.data, src.shape[0], scratch.data_ptr(), repeats,
                                   ctypes.byref(best), ctypes.byref(ms), _stream_handle(stream)), "atos_autotune")
        return best, ms.value

    def timeline(self, bucket_us: float = 0.0, nbuckets: int = 0):
        """Records the throughput timeline of the following calls (nbuckets buckets of bucket_us
        microseconds from each call's start); timeline() turns it off."""
        _check(lib().atos_timeline(self._h, int(bucket_us * 1000), int(nbuckets)), "atos_timeline")
        self._tl_buckets = int(nbuckets)

    def timeline_read(self):
        """(tasks, edges) per bucket of the last call, as int64 numpy arrays."""
        nb = getattr(self, "_tl_buckets", 0)
        tasks = np.zeros(nb, np.int64)
        edges = np.zeros(nb, np.int64)
        _check(lib().atos_timeline_read(self._h, tasks.ctypes.data, edges.ctypes.data, nb), "atos_timeline_read")
        return tasks, edges

    def edge_ceiling(self, kind: str = "scatter", repeats: int = 3, stream=None, spread_ids: bool = False) -> float:
        """Device ms of one ideal pass over every CSR entry ("scatter": red.add into state[col[e]],
        "gather": a load of state[col[e]]), with no scheduler: the edge-loop roofline (on the
        spread-id copy of the graph when ``spread_ids``)."""
        ms = ctypes.c_double(0)
        code = {"scatter": 0, "gather": 1}[kind] | (2 if spread_ids else 0)
        _check(lib().atos_edge_ceiling(self._h, code, repeats, ctypes.byref(ms), _stream_handle(stream)),
               "atos_edge_ceiling")
        return ms.value

    def tuned_config(self, app: str):
        """The cached tuned Config for this graph's class, or None if the class was not tuned."""
        code = {"bfs": APP_BFS, "pagerank": APP_PAGERANK, "color": APP_COLOR}[app]
        cfg = Config()
        rc = lib().atos_tuned_config(self._h, code, ctypes.byref(cfg))
        return cfg if rc == OK else None

    # ------------------------------------------------------------------------------ apps

    def bfs(self, sources, depths=None, cfg: Config | None = None, stream=None, stats: bool = True):
        """Hop distances from each source: returns (depths [len(sources), n] int32 CUDA tensor,
        Stats or None).  Raises AtosError on failure (including device-side errors when stats)."""
        import torch
        src = np.ascontiguousarray(np.atleast_1d(np.asarray(sources)), dtype=np.int32)
        if depths is None:
            depths = torch.empty((src.shape[0], self.n), dtype=torch.int32, device="cuda")
        st = Stats() if stats else None
        rc = lib().atos_bfs(self._h, src.ctypes.data, src.shape[0], depths.data_ptr(),
                            ctypes.byref(cfg) if cfg is not None else None, _stream_handle(stream),
                            ctypes.byref(st) if st is not None else None)
        _check(rc, "atos_bfs")
        return depths, st

    def pagerank(self, alpha: float = 0.85, eps: float = 1e-9, rank=None, cfg: Config | None = None, stream=None,
                 stats: bool = True):
        """Push-residual PageRank: returns (rank [n] float32 CUDA tensor summing to 1, Stats)."""
        import torch
        if rank is None:
            rank = torch.empty(self.n, dtype=torch.float32, device="cuda")
        st = Stats() if stats else None
        rc = lib().atos_pagerank(self._h, float(alpha), float(eps), rank.data_ptr() if self.n else None,
                                 ctypes.byref(cfg) if cfg is not None else None, _stream_handle(stream),
                                 ctypes.byref(st) if st is not None else None)
        _check(rc, "atos_pagerank")
        return rank, st

    def color(self, colors=None, cfg: Config | None = None, stream=None, stats: bool = True):
        """Speculative greedy colouring: returns (colors [n] int32 CUDA tensor, num_colors, Stats)."""
        import torch
        if colors is None:
            colors = torch.empty(self.n, dtype=torch.int32, device="cuda")
        st = Stats() if stats else None
        k = ctypes.c_int32(0)
        rc = lib().atos_color(self._h, colors.data_ptr() if self.n else None, ctypes.byref(k) if stats else None,
                              ctypes.byref(cfg) if cfg is not None else None, _stream_handle(stream),
                              ctypes.byref(st) if st is not None else None)
        _check(rc, "atos_color")
        return colors, (k.value if stats else None), st


def _instance_table(graphs, specs):
    """(atos_instance array, output tensors) for batch specs (see Batch)."""
    import torch
    arr = (Instance * len(specs))()
    outputs = []
    for i, spec in enumerate(specs):
        kind, gi = spec[0], int(spec[1])
        n = graphs[gi].n if 0 <= gi < len(graphs) else 1  # a bad index is the C ABI's to reject
        q = arr[i]
        q.graph = gi
        if kind == "bfs":
            q.app, q.source = APP_BFS, int(spec[2])
            out = torch.empty(n, dtype=torch.int32, device="cuda")
        elif kind == "pagerank":
            q.app = APP_PAGERANK
            q.alpha = float(spec[2]) if len(spec) > 2 else 0.85
            q.eps = float(spec[3]) if len(spec) > 3 else 1e-9
            out = torch.empty(n, dtype=torch.float32, device="cuda")
        elif kind == "color":
            q.app = APP_COLOR
            out = torch.empty(n, dtype=torch.int32, device="cuda")
        else:
            raise ValueError(kind)
        q.out = out.data_ptr()
        outputs.append(out)
    return arr, outputs


def batch_autotune(graphs, specs, repeats: int = 1, stream=None):
    """Times candidate configurations (worker, fetch, window, persistent vs discrete, PageRank
    enqueue rule) of a batch of ``specs`` over ``graphs``; returns (best Config, device ms)."""
    graphs = list(graphs)
    arr, outputs = _instance_table(graphs, list(specs))
    handles = (ctypes.c_void_p * len(graphs))(*[g._h.value for g in graphs])
    best, ms = Config(), ctypes.c_double(0)
    _check(lib().atos_batch_autotune(handles, len(graphs), arr, len(specs), repeats, ctypes.byref(best),
                                     ctypes.byref(ms), _stream_handle(stream)), "atos_batch_autotune")
    del outputs
    return best, ms.value


class Batch:
    """Many instances over several graphs in one persistent launch (wraps an atos_batch_t).

    ``specs`` is a list of ("bfs", graph_index, source), ("pagerank", graph_index[, alpha, eps])
    or ("color", graph_index); an output tensor is allocated for each instance (``outputs``).
    The graphs must stay open while the batch lives."""

    def __init__(self, graphs, specs, cfg: Config | None = None):
        self._h = ctypes.c_void_p()
        self.graphs = list(graphs)
        self.specs = list(specs)
        arr, self.outputs = _instance_table(self.graphs, self.specs)
        handles = (ctypes.c_void_p * len(self.graphs))(*[g._h.value for g in self.graphs])
        _check(lib().atos_batch_create(handles, len(self.graphs), arr, len(self.specs),
                                       ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(self._h)),
               "atos_batch_create")
        ni, w, grid = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        lib().atos_batch_info(self._h, ctypes.byref(ni), ctypes.byref(w), ctypes.byref(grid))
        self.window, self.grid = w.value, grid.value

    def run(self, stream=None, graph: bool = False):
        fn = lib().atos_batch_run_graph if graph else lib().atos_batch_run
        _check(fn(self._h, _stream_handle(stream)), "atos_batch_run")

    def stats(self, stream=None):
        total = Stats()
        per = (Stats * len(self.specs))()
        rc = lib().atos_batch_stats(self._h, ctypes.byref(total), per, _stream_handle(stream))
        _check(rc, "atos_batch_stats")
        return total, list(per)

    def close(self):
        if self._h:
            lib().atos_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching request server over resident graphs (wraps an atos_server_t).

    ``submit`` admits a request now if a slot and arena memory are free (else returns None);
    ``step`` runs one epoch (a persistent launch bounded by ``slice_ns``) over every admitted
    request; ``poll`` returns the completion records."""

    def __init__(self, graphs, max_slots: int = 64, budget_bytes: int = 8 << 30, cfg: Config | None = None):
        self._h = ctypes.c_void_p()
        self.graphs = list(graphs)
        handles = (ctypes.c_void_p * len(self.graphs))(*[g._h.value for g in self.graphs])
        _check(lib().atos_server_create(handles, len(self.graphs), max_slots, int(budget_bytes),
                                        ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(self._h)),
               "atos_server_create")
        self._outputs = {}

    def submit(self, kind: str, graph: int, source: int = 0, alpha: float = 0.85, eps: float = 1e-9, out=None):
        """Returns (request id, output tensor), or None when the request cannot be admitted now."""
        import torch
        n = self.graphs[graph].n
        q = Instance()
        q.graph = graph
        if kind == "bfs":
            q.app, q.source = APP_BFS, int(source)
            out = out if out is not None else torch.empty(n, dtype=torch.int32, device="cuda")
        elif kind == "pagerank":
            q.app, q.alpha, q.eps = APP_PAGERANK, float(alpha), float(eps)
            out = out if out is not None else torch.empty(n, dtype=torch.float32, device="cuda")
        elif kind == "color":
            q.app = APP_COLOR
            out = out if out is not None else torch.empty(n, dtype=torch.int32, device="cuda")
        else:
            raise ValueError(kind)
        q.out = out.data_ptr()
        rid = ctypes.c_int64(-1)
        rc = lib().atos_server_submit(self._h, ctypes.byref(q), ctypes.byref(rid))
        if rc == ERR_BUSY:
            return None
        _check(rc, "atos_server_submit")
        self._outputs[rid.value] = out
        return rid.value, out

    def step(self, slice_ns: int = 1_000_000) -> int:
        left = ctypes.c_int32(0)
        _check(lib().atos_server_step(self._h, int(slice_ns), ctypes.byref(left)), "atos_server_step")
        return left.value

    def poll(self, max_records: int = 4096):
        buf = (Completion * max_records)()
        cnt = ctypes.c_int32(0)
        _check(lib().atos_server_poll(self._h, buf, max_records, ctypes.byref(cnt)), "atos_server_poll")
        out = []
        for c in buf[:cnt.value]:
            d = c.as_dict()
            d["out"] = self._outputs.pop(c.id, None)
            out.append(d)
        return out

    def info(self):
        a, used, size, ep = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().atos_server_info(self._h, ctypes.byref(a), ctypes.byref(used), ctypes.byref(size),
                                      ctypes.byref(ep)), "atos_server_info")
        return {"active": a.value, "arena_used": used.value, "arena_size": size.value, "epochs": ep.value}

    def close(self):
        if self._h:
            lib().atos_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
