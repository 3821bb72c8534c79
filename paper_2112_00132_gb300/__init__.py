"""GB300 (sm_103a) task-parallel dynamic scheduler for irregular graph work.

A persistent-kernel (or discrete-launch) device worklist with warp- or CTA-sized workers and a
tunable fetch size, driving speculative BFS, asynchronous push-residual PageRank and speculative
greedy colouring on int32 CSR graphs (the Atos model, Chen et al., PPoPP 2022).  The compute is
in ``libatos.so`` (hand-written CUDA behind the C ABI of ``include/atos.h``); this package is the
Python binding.
"""
from ._binding import (  # noqa: F401
    BSP, DISCRETE, FETCH_FIXED, FETCH_GREEDY, FETCH_SPREAD, FLAG_PHANTOM_TASK, FLAG_PR_CROSSING, FLAG_SPREAD_IDS, FLAG_GC_ORDERED, FLAG_BFS_EXPAND_ONCE, FLAG_BSP_DEVICE_LOOP, FLAG_BSP_PER_SOURCE, FLAG_GC_DEPENDENCY, FLAG_BFS_SPLIT_ROWS, PERSISTENT, UNREACHED, WORKER_WARP, WORKER_THREAD,
    AtosError, Batch, Completion, batch_autotune, Config, Graph, Instance, Server, Stats, csr_validate, header_functions, kernel_launches, lib, queue_config, status_string,
    version,
)
from . import _binding as abi  # noqa: F401


def build(force: bool = False) -> str:
    """Compiles libatos.so for sm_103a (nvcc) and returns its path."""
    from .compile_lib import build as _build
    return _build(force=force)
