"""Bounded waits and error paths on the GPU, made to fail on the host side without faulting
anything: a task that is counted but never pushed (the workers' waits run out and report
ATOS_ERR_TIMEOUT), and a ring too small for a single worker (ATOS_ERR_QUEUE_OVERFLOW).  After each
failure the same graph object must run correctly again."""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_common import atos_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def atos():
    return atos_lib()


@pytest.mark.parametrize("worker", [32, 256])
def test_phantom_task_times_out_then_recovers(atos, worker):
    g = gg.rmat(10, 16, seed=2)
    ref = oracle.bfs(g, 0)
    with atos.Graph.from_csr(g) as G:
        cfg = atos.queue_config(worker_size=worker, fetch_size=32 if worker == 32 else 256,
                                flags=atos.FLAG_PHANTOM_TASK, spin_limit_ns=20_000_000)
        with pytest.raises(atos.AtosError) as e:
            G.bfs([0], cfg=cfg)
        assert e.value.status == atos.abi.ERR_TIMEOUT
        depths, st = G.bfs([0])
        assert st.status == 0 and np.array_equal(depths.cpu().numpy()[0], ref)


def test_small_ring_overflows_then_recovers(atos):
    g = gg.rmat(12, 16, seed=1)  # vertex 0 has more than 1024 neighbours
    ref = oracle.bfs(g, 0)
    with atos.Graph.from_csr(g) as G:
        cfg = atos.queue_config(num_blocks=1, queue_capacity=1024)
        with pytest.raises(atos.AtosError) as e:
            G.bfs([0], cfg=cfg)
        assert e.value.status == atos.abi.ERR_QUEUE_OVERFLOW
        depths, st = G.bfs([0])
        assert st.status == 0 and np.array_equal(depths.cpu().numpy()[0], ref)
        # colouring with a ring smaller than the graph, one worker: the check tasks overflow
        with pytest.raises(atos.AtosError) as e:
            G.color(cfg=atos.queue_config(num_blocks=1, queue_capacity=1024))
        assert e.value.status == atos.abi.ERR_QUEUE_OVERFLOW
        colors, k, st = G.color()
        assert oracle.check_coloring(g, colors.cpu().numpy())[0] == 0


def test_malformed_csr_rejected_on_host(atos):
    g = gg.path(6)
    bad = g.col.copy()
    bad[2] = 99
    with pytest.raises(atos.AtosError) as e:
        atos.Graph(g.row_ptr, bad)
    assert e.value.status == atos.abi.ERR_BAD_CSR
    with pytest.raises(atos.AtosError) as e:
        atos.Graph(np.array([0, 1, 1]), np.array([1]), check_symmetric=True)
    assert e.value.status == atos.abi.ERR_BAD_CSR


def test_edge_ceiling_probe(atos):
    g = gg.rmat(12, 16, seed=1)
    with atos.Graph.from_csr(g) as G:
        for kind in ("scatter", "gather"):
            for spread in (False, True):
                ms = G.edge_ceiling(kind, repeats=2, spread_ids=spread)
                assert ms > 0
        rc = atos.abi.lib().atos_edge_ceiling(G._h, 9, 1, ctypes.byref(ctypes.c_double()), None)
        assert rc == atos.abi.ERR_INVALID_ARG
    with atos.Graph.from_csr(gg.from_edges(3, [], "isolated3")) as G:
        assert G.edge_ceiling("scatter") == 0.0
