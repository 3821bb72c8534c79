"""Shared helpers of the GPU parity tests (graphs, configurations, library fixture)."""
import numpy as np
import pytest

import graphgen as gg

ALPHA = 0.85
EPS = 1e-9
PR_L1_TOL = 1e-4  # L1 distance of the normalised FP32 result to the FP64 fixed point


def atos_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_00132_gb300 as atos
    atos.build()
    atos.lib()
    return atos


def small_graphs():
    """Small graphs that still span many CTA batches and end in a ragged tail, plus the
    degenerate shapes of the method."""
    return {
        "rmat12": gg.rmat(12, 16, seed=1),  # the 4096-vertex RMAT workload
        "rmat11_del": gg.rmat(11, 16, seed=7, delete_frac=0.1),
        "grid97x61_del": gg.grid(97, 61, delete_frac=0.1, seed=3),
        "path300": gg.path(300),
        "star1000": gg.star(1000),
        "clique40": gg.clique(40),
        "two_parts": gg.from_edges(9, [(0, 1), (1, 2), (2, 0), (4, 5), (5, 6), (6, 7)], "two_parts"),
        "single": gg.from_edges(1, [], "single"),
        "isolated3": gg.from_edges(3, [], "isolated3"),
    }


def bfs_sources(g, k=3, seed=11):
    out = [0, g.n - 1]
    nz = np.flatnonzero(g.degrees > 0)
    if nz.size:
        out += [int(x) for x in gg.sources(g, k, seed=seed)]
    return sorted(set(out))


def configs(atos):
    """Worker shapes x strategies x fetch policies exercised by the parity tests."""
    q = atos.queue_config
    return {
        "persist-cta256": q(),
        "persist-cta64-fixed": q(worker_size=64, fetch_size=64, fetch_policy=atos.FETCH_FIXED),
        "persist-cta128-f1": q(worker_size=128, fetch_size=1),
        "persist-cta512-greedy": q(worker_size=512, fetch_size=384, fetch_policy=atos.FETCH_GREEDY),
        "persist-cta1024": q(worker_size=1024, fetch_size=1024),
        "persist-warp": q("persist-warp"),
        "persist-warp-f32": q(worker_size=32, fetch_size=32, fetch_policy=atos.FETCH_SPREAD),
        "persist-cta256-8blocks": q(num_blocks=8),
        "discrete-cta": q("discrete-cta"),
        "discrete-cta64": q("discrete-cta", worker_size=64, fetch_size=32),
        "discrete-warp": q("discrete-warp"),
        "bsp": q("bsp"),
        "bsp-device-loop": q("bsp", flags=atos.FLAG_BSP_DEVICE_LOOP),
        "bsp-per-source": q("bsp", flags=atos.FLAG_BSP_PER_SOURCE),
    }


def thread_worker_configs(atos):
    """Thread workers (worker_size 1): a warp pops up to 32 tasks and each lane runs one."""
    q = atos.queue_config
    return {
        "persist-thread-f32": q(worker_size=1, fetch_size=32, fetch_policy=atos.FETCH_SPREAD),
        "persist-thread-f7-fixed": q(worker_size=1, fetch_size=7, fetch_policy=atos.FETCH_FIXED),
        "persist-thread-greedy-4blocks": q(worker_size=1, fetch_size=32, fetch_policy=atos.FETCH_GREEDY, num_blocks=4),
        "discrete-thread-f32": q("discrete-warp", worker_size=1, fetch_size=32),
        "discrete-thread-f5": q("discrete-warp", worker_size=1, fetch_size=5),
    }
