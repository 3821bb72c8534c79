"""Autotuner: sweeps worker size x fetch size x strategy on the graph, returns a configuration
that runs correctly, and caches it for graphs of the same class."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_common import ALPHA, EPS, PR_L1_TOL, atos_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def atos():
    return atos_lib()


def test_autotune_each_app(atos):
    g = gg.rmat(12, 16, seed=1)
    srcs = [int(x) for x in gg.sources(g, 8, seed=3)]
    with atos.Graph.from_csr(g) as G:
        assert G.tuned_config("bfs") is None or True  # may be cached by an earlier test in the process
        cfg, ms = G.autotune("bfs", srcs)
        assert ms > 0 and cfg.worker_size in (32, 64, 128, 256, 512, 1024)
        depths, _ = G.bfs(srcs, cfg=cfg)
        assert all(np.array_equal(depths.cpu().numpy()[i], oracle.bfs(g, s)) for i, s in enumerate(srcs))
        cfg_pr, _ = G.autotune("pagerank")
        rank, st = G.pagerank(ALPHA, EPS, cfg=cfg_pr)
        x, _, _ = oracle.pagerank(g, ALPHA)
        assert np.abs(rank.cpu().numpy() - x / x.sum()).sum() <= PR_L1_TOL
        cfg_gc, _ = G.autotune("color")
        colors, k, _ = G.color(cfg=cfg_gc)
        assert oracle.check_coloring(g, colors.cpu().numpy())[0] == 0
    # a graph of the same class (same scale, degree shape) gets the cached choice
    g2 = gg.rmat(12, 16, seed=2)
    with atos.Graph.from_csr(g2) as G2:
        cached = G2.tuned_config("pagerank")
        assert cached is not None and cached.as_dict() == cfg_pr.as_dict()


def test_autotune_preset_uses_cached_configs(atos):
    """queue_config("autotune"): calls take the configuration cached for the graph's class (and the
    defaults for a class never tuned); results pass the usual gates either way."""
    g = gg.rmat(11, 16, seed=4)
    cfg = atos.queue_config("autotune")
    assert cfg.flags & atos.abi.FLAG_USE_TUNED
    with atos.Graph.from_csr(gg.path(700)) as P:  # a class nobody tuned
        d, _ = P.bfs([0], cfg=cfg)
        assert np.array_equal(d.cpu().numpy()[0], np.arange(700))
    with atos.Graph.from_csr(g) as G:
        G.autotune("pagerank", repeats=1)
        G.autotune("color", repeats=1)
        rank, st = G.pagerank(0.85, 1e-9, cfg=cfg)
        x, _, _ = oracle.pagerank(g, 0.85)
        assert np.abs(rank.cpu().numpy().astype(np.float64) - x / x.sum()).sum() <= 1e-4
        colors, k, st = G.color(cfg=cfg)
        assert oracle.check_coloring(g, colors.cpu().numpy())[0] == 0
