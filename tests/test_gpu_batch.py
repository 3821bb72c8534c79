"""Batched launches: many instances (BFS sources, PageRanks, colourings) over several graphs in one
persistent launch, and its CUDA-graph replay.  Each instance's result must be the same alone and
in the mix: BFS depths bit-exact, PageRank within the L1 tolerance of the oracle, colourings
proper."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_common import ALPHA, EPS, PR_L1_TOL, atos_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def atos():
    return atos_lib()


@pytest.fixture(scope="module")
def graphs():
    return [gg.rmat(11, 16, seed=3), gg.grid(60, 41, delete_frac=0.1, seed=4), gg.rmat(10, 16, seed=5, delete_frac=0.1),
            gg.path(200)]


def mixed_specs(graphs, per_graph_bfs=3):
    specs = []
    for gi, g in enumerate(graphs):
        for s in gg.sources(g, per_graph_bfs, seed=gi + 1):
            specs.append(("bfs", gi, int(s)))
        specs.append(("pagerank", gi, ALPHA, EPS))
        specs.append(("color", gi))
    return specs


def check_results(graphs, specs, outputs, per):
    for (kind, gi, *rest), out, st in zip(specs, outputs, per):
        g = graphs[gi]
        res = out.cpu().numpy()
        assert st.status == 0
        if kind == "bfs":
            assert np.array_equal(res, oracle.bfs(g, rest[0])), f"bfs graph {gi} source {rest[0]}"
        elif kind == "pagerank":
            x, _, _ = oracle.pagerank(g, ALPHA)
            l1 = np.abs(res.astype(np.float64) - x / x.sum()).sum()
            assert l1 <= PR_L1_TOL, f"pagerank graph {gi}: L1 {l1}"
            assert l1 <= st.error_bound * 1.0001 + 1e-9  # the FP64 certificate covers the FP32 output
        else:
            code, bad, k = oracle.check_coloring(g, res)
            assert code == 0 and k == st.num_colors, f"colouring graph {gi}: code {code} vertex {bad}"


@pytest.mark.parametrize("worker,window", [(256, 0), (256, 1), (256, 3), (128, 100), (32, 4), (512, 2)])
def test_mixed_batch_matches_oracle(atos, graphs, worker, window):
    Gs = [atos.Graph.from_csr(g) for g in graphs]
    specs = mixed_specs(graphs)
    cfg = atos.queue_config(worker_size=worker, fetch_size=32 if worker == 32 else worker, window=window)
    with atos.Batch(Gs, specs, cfg) as B:
        B.run()
        total, per = B.stats()
        assert total.status == 0
        check_results(graphs, specs, B.outputs, per)
    for G in Gs:
        G.close()


def test_batch_cuda_graph_replay(atos, graphs):
    import torch
    Gs = [atos.Graph.from_csr(g) for g in graphs]
    specs = mixed_specs(graphs, per_graph_bfs=2)
    with atos.Batch(Gs, specs) as B:
        B.run(graph=True)
        total, per = B.stats()
        check_results(graphs, specs, B.outputs, per)
        for out in B.outputs:
            out.fill_(-5)
        l0 = atos.kernel_launches()
        B.run(graph=True)  # replay of the captured graph recomputes everything
        assert atos.kernel_launches() > l0  # a replay counts the library kernels it runs
        total, per = B.stats()
        check_results(graphs, specs, B.outputs, per)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            B.run(stream=stream, graph=True)
        total, per = B.stats(stream=stream)
        check_results(graphs, specs, B.outputs, per)
    for G in Gs:
        G.close()


def test_same_alone_and_in_the_mix(atos, graphs):
    Gs = [atos.Graph.from_csr(g) for g in graphs]
    specs = mixed_specs(graphs, per_graph_bfs=2)
    with atos.Batch(Gs, specs) as B:
        B.run()
        B.stats()
        for (kind, gi, *rest), out in zip(specs, B.outputs):
            G = Gs[gi]
            if kind == "bfs":
                alone, _ = G.bfs([rest[0]])
                assert np.array_equal(alone.cpu().numpy()[0], out.cpu().numpy())
            elif kind == "pagerank":
                alone, _ = G.pagerank(ALPHA, EPS)
                assert np.abs(alone.cpu().numpy().astype(np.float64) - out.cpu().numpy()).sum() <= 2 * PR_L1_TOL
            else:
                alone, k, _ = G.color()
                assert oracle.check_coloring(graphs[gi], alone.cpu().numpy())[0] == 0
                assert oracle.check_coloring(graphs[gi], out.cpu().numpy())[0] == 0
    for G in Gs:
        G.close()


def test_batch_invalid(atos, graphs):
    G = atos.Graph.from_csr(graphs[0])
    for bad in ([("bfs", 1, 0)], [("bfs", 0, graphs[0].n)], [("pagerank", 0, 1.5, EPS)]):
        with pytest.raises(atos.AtosError) as e:
            atos.Batch([G], bad)
        assert e.value.status == atos.abi.ERR_INVALID_ARG
    with pytest.raises(atos.AtosError) as e:
        atos.Batch([G], [("bfs", 0, 0)], atos.queue_config("bsp"))
    assert e.value.status == atos.abi.ERR_UNSUPPORTED
    with pytest.raises(atos.AtosError) as e:  # a thread worker fetches at most 32 tasks
        atos.Batch([G], [("bfs", 0, 0)], atos.queue_config(worker_size=1, fetch_size=64))
    assert e.value.status == atos.abi.ERR_INVALID_ARG
    with atos.Batch([G], [("bfs", 0, 0)], atos.queue_config("discrete-cta")) as B:
        with pytest.raises(atos.AtosError) as e:  # host-driven generations cannot be captured
            B.run(graph=True)
        assert e.value.status == atos.abi.ERR_UNSUPPORTED
    G.close()


@pytest.mark.parametrize("worker", [256, 1024, 32])
def test_mixed_batch_pagerank_crossing(atos, graphs, worker):
    """The threshold-crossing PageRank variant inside a mixed batch: per-instance results unchanged."""
    Gs = [atos.Graph.from_csr(g) for g in graphs]
    specs = mixed_specs(graphs, per_graph_bfs=2)
    cfg = atos.queue_config(worker_size=worker, fetch_size=32 if worker == 32 else worker,
                            flags=atos.FLAG_PR_CROSSING)
    with atos.Batch(Gs, specs, cfg) as B:
        B.run(graph=True)
        total, per = B.stats()
        assert total.status == 0
        check_results(graphs, specs, B.outputs, per)
    for G in Gs:
        G.close()


@pytest.mark.parametrize("preset,worker", [("discrete-cta", 256), ("discrete-cta", 64), ("discrete-warp", 32)])
def test_discrete_batch_matches_oracle(atos, graphs, preset, worker):
    """The discrete strategy over a mixed batch: one launch per generation of every instance."""
    Gs = [atos.Graph.from_csr(g) for g in graphs]
    specs = mixed_specs(graphs, per_graph_bfs=2)
    cfg = atos.queue_config(preset, worker_size=worker, fetch_size=min(worker, 32) if worker <= 64 else worker)
    with atos.Batch(Gs, specs, cfg) as B:
        B.run()
        total, per = B.stats()
        assert total.status == 0
        check_results(graphs, specs, B.outputs, per)
    for G in Gs:
        G.close()


def test_batch_autotune(atos, graphs):
    Gs = [atos.Graph.from_csr(g) for g in graphs]
    specs = mixed_specs(graphs, per_graph_bfs=2)
    cfg, ms = atos.batch_autotune(Gs, specs, repeats=1)
    assert ms > 0 and cfg.worker_size in (32, 64, 128, 256, 512, 1024)
    with atos.Batch(Gs, specs, cfg) as B:
        B.run(graph=cfg.strategy == atos.PERSISTENT)
        total, per = B.stats()
        check_results(graphs, specs, B.outputs, per)
    for G in Gs:
        G.close()


@pytest.mark.parametrize("preset,worker", [(None, 256), (None, 1024), ("discrete-cta", 256), (None, 32)])
def test_mixed_batch_spread_ids(atos, graphs, preset, worker):
    """PageRank and colouring instances on their graphs' spread-id copies inside a batch: results in
    the caller's ids, the same gates; BFS instances of the same batch unaffected."""
    Gs = [atos.Graph.from_csr(g) for g in graphs]
    specs = mixed_specs(graphs, per_graph_bfs=2)
    cfg = atos.queue_config(preset, worker_size=worker, fetch_size=32 if worker == 32 else worker,
                            flags=atos.FLAG_SPREAD_IDS)
    with atos.Batch(Gs, specs, cfg) as B:
        B.run(graph=cfg.strategy == atos.PERSISTENT)
        total, per = B.stats()
        assert total.status == 0
        check_results(graphs, specs, B.outputs, per)
    for G in Gs:
        G.close()
