"""Serving: requests over resident graphs, admitted by footprint, run in epochs that pause and
resume their workers; every result must equal the same request run alone (BFS bit-exact,
PageRank within the L1 tolerance, colouring proper), also for requests admitted while others are
in flight and for requests that span many epochs."""
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
    return [gg.rmat(12, 16, seed=1), gg.grid(80, 61, delete_frac=0.1, seed=2), gg.rmat(11, 16, seed=9, delete_frac=0.1)]


def check(graph, kind, source, out):
    res = out.cpu().numpy()
    if kind == "bfs":
        return np.array_equal(res, oracle.bfs(graph, source))
    if kind == "pagerank":
        x, _, _ = oracle.pagerank(graph, ALPHA)
        return np.abs(res.astype(np.float64) - x / x.sum()).sum() <= PR_L1_TOL
    return oracle.check_coloring(graph, res)[0] == 0


def drain(S, slice_ns, limit=100000):
    done = []
    for _ in range(limit):
        left = S.step(slice_ns)
        done += S.poll()
        if left == 0:
            break
    return done


def test_server_mixed_requests_match_oracle(atos, graphs):
    Gs = [atos.Graph.from_csr(g) for g in graphs]
    reqs = {}
    with atos.Server(Gs, max_slots=32, budget_bytes=2 << 30) as S:
        for gi, g in enumerate(graphs):
            for s in gg.sources(g, 3, seed=gi + 7):
                rid, out = S.submit("bfs", gi, int(s))
                reqs[rid] = ("bfs", gi, int(s))
            rid, _ = S.submit("pagerank", gi, alpha=ALPHA, eps=EPS)
            reqs[rid] = ("pagerank", gi, 0)
            rid, _ = S.submit("color", gi)
            reqs[rid] = ("color", gi, 0)
        done = drain(S, 200_000)
        assert sorted(d["id"] for d in done) == sorted(reqs)
        for d in done:
            kind, gi, src = reqs[d["id"]]
            assert d["status"] == 0
            assert check(graphs[gi], kind, src, d["out"]), (kind, gi, src, d)
            if kind == "pagerank":  # the completion's FP64 certificate covers the actual distance
                x, _, _ = oracle.pagerank(graphs[gi], ALPHA)
                l1 = np.abs(d["out"].cpu().numpy().astype(np.float64) - x / x.sum()).sum()
                assert 0 < d["error_bound"] <= PR_L1_TOL and l1 <= d["error_bound"] * 1.0001 + 1e-9
        assert S.info()["arena_used"] == 0 and S.info()["active"] == 0
    for G in Gs:
        G.close()


def test_server_admits_while_others_are_in_flight(atos, graphs):
    Gs = [atos.Graph.from_csr(g) for g in graphs]
    with atos.Server(Gs, max_slots=16, budget_bytes=2 << 30) as S:
        first = [S.submit("pagerank", 0), S.submit("color", 2)]
        left = S.step(50_000)  # a short slice: the PageRank is still in flight
        assert left >= 1
        late = [S.submit("bfs", 1, 0), S.submit("bfs", 0, 5), S.submit("pagerank", 2)]
        done = S.poll() + drain(S, 100_000)
        ids = {d["id"]: d for d in done}
        kinds = {first[0][0]: ("pagerank", 0, 0), first[1][0]: ("color", 2, 0), late[0][0]: ("bfs", 1, 0),
                 late[1][0]: ("bfs", 0, 5), late[2][0]: ("pagerank", 2, 0)}
        assert set(ids) == set(kinds)
        for rid, (kind, gi, src) in kinds.items():
            assert check(graphs[gi], kind, src, ids[rid]["out"]), (kind, gi)
        assert max(d["epochs"] for d in done) > 1
    for G in Gs:
        G.close()


def test_server_result_same_alone_and_in_the_mix(atos, graphs):
    G = atos.Graph.from_csr(graphs[0])
    alone_bfs, _ = G.bfs([17])
    alone_pr, _ = G.pagerank(ALPHA, EPS)
    with atos.Server([G], max_slots=8, budget_bytes=1 << 30) as S:
        rb = S.submit("bfs", 0, 17)
        rp = S.submit("pagerank", 0)
        for s in (3, 99, 1024):
            S.submit("bfs", 0, s)
        S.submit("color", 0)
        done = {d["id"]: d for d in drain(S, 30_000)}
        assert np.array_equal(done[rb[0]]["out"].cpu().numpy(), alone_bfs.cpu().numpy()[0])
        assert np.abs(done[rp[0]]["out"].cpu().numpy() - alone_pr.cpu().numpy()).sum() <= 2 * PR_L1_TOL
    G.close()


def test_server_admission_by_footprint(atos, graphs):
    G = atos.Graph.from_csr(graphs[0])
    with atos.Server([G], max_slots=8, budget_bytes=24 << 20) as S:  # room for about two requests
        got = [S.submit("bfs", 0, s) for s in range(6)]
        admitted = [x for x in got if x is not None]
        assert 1 <= len(admitted) < 6 and got[-1] is None
        drain(S, 1_000_000)
        assert S.info()["arena_used"] == 0
        assert S.submit("bfs", 0, 5) is not None  # memory came back
        drain(S, 1_000_000)
    G.close()


def test_server_rejects_warp_hosted_workers(atos, graphs):
    """Serving pauses CTA workers between epochs; warp and thread workers are not offered."""
    G = atos.Graph.from_csr(graphs[0])
    for w in (1, 32):
        with pytest.raises(atos.AtosError) as e:
            atos.Server([G], max_slots=4, budget_bytes=8 << 20, cfg=atos.queue_config(worker_size=w, fetch_size=32))
        assert e.value.status == atos.abi.ERR_UNSUPPORTED
    G.close()


def test_serving_loop_short_run(atos, graphs):
    """The Poisson serving loop: every request completes, latencies are reported, and sampled
    results are correct."""
    from paper_2112_00132_gb300 import serve
    res = serve.serve(graphs, rate=400.0, duration=1.5, warmup=0.3, slice_ns=500_000, max_slots=64,
                      budget_bytes=4 << 30, keep=40)
    assert res["unfinished"] == 0 and res["completed"] == res["requests"] > 100
    assert res["p50_ms"] is not None and res["p99_ms"] >= res["p50_ms"] > 0
    for r in res["kept"]:
        assert check(graphs[r["graph"]], r["kind"], r["source"], r["out"]), r["kind"]


def test_server_spread_ids(atos, graphs):
    """A server whose PageRank and colouring requests run on the graphs' spread-id copies."""
    Gs = [atos.Graph.from_csr(g) for g in graphs]
    reqs = {}
    cfg = atos.queue_config(flags=atos.FLAG_SPREAD_IDS)
    with atos.Server(Gs, max_slots=16, budget_bytes=2 << 30, cfg=cfg) as S:
        for gi, g in enumerate(graphs):
            rid, _ = S.submit("pagerank", gi, alpha=ALPHA, eps=EPS)
            reqs[rid] = ("pagerank", gi, 0)
            rid, _ = S.submit("color", gi)
            reqs[rid] = ("color", gi, 0)
            src = int(gg.sources(g, 1, seed=gi + 3)[0])
            rid, _ = S.submit("bfs", gi, src)
            reqs[rid] = ("bfs", gi, src)
        done = drain(S, 200_000)
        assert sorted(d["id"] for d in done) == sorted(reqs)
        for d in done:
            kind, gi, src = reqs[d["id"]]
            assert d["status"] == 0 and check(graphs[gi], kind, src, d["out"]), (kind, gi, src, d)
            if kind == "pagerank":
                x, _, _ = oracle.pagerank(graphs[gi], ALPHA)
                l1 = np.abs(d["out"].cpu().numpy().astype(np.float64) - x / x.sum()).sum()
                assert l1 <= d["error_bound"] * 1.0001 + 1e-9
        assert S.info()["arena_used"] == 0
    for G in Gs:
        G.close()
