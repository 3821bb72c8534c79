"""Host logic of the serving loop on the CPU, with a fake server in place of the GPU one: Poisson
arrivals, the two admission queues (at most `max_large` requests on large graphs in flight, no
head-of-line blocking of small requests behind them), and latency accounting."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
from paper_2112_00132_gb300 import serve  # noqa: E402
from paper_2112_00132_gb300._binding import Config  # noqa: E402


class FakeGraph:
    def __init__(self, n):
        self.n = n


class FakeServer:
    """Admits up to max_slots requests; a request finishes after a fixed number of epochs
    (long on large graphs)."""

    def __init__(self, graphs, max_slots, large_n, steps_small=2, steps_large=40):
        self.graphs, self.max_slots, self.large_n = graphs, max_slots, large_n
        self.steps_small, self.steps_large = steps_small, steps_large
        self.active = {}
        self.done = []
        self.next_id = 0
        self.epochs = 0
        self.max_large_seen = 0

    def submit(self, kind, graph, source=0, alpha=0.85, eps=1e-9):
        if len(self.active) >= self.max_slots:
            return None
        rid = self.next_id
        self.next_id += 1
        large = self.graphs[graph].n > self.large_n
        self.active[rid] = [self.steps_large if large else self.steps_small, kind, graph, large]
        self.max_large_seen = max(self.max_large_seen, sum(1 for a in self.active.values() if a[3]))
        return rid, None

    def step(self, slice_ns):
        self.epochs += 1
        for rid in list(self.active):
            self.active[rid][0] -= 1
            if self.active[rid][0] <= 0:
                _, kind, graph, _ = self.active.pop(rid)
                self.done.append({"id": rid, "status": 0, "edges": 10, "error_bound": 0.0, "out": None})
        return len(self.active)

    def poll(self):
        out, self.done = self.done, []
        return out

    def info(self):
        return {"epochs": self.epochs, "active": len(self.active)}

    def close(self):
        pass


def test_poisson_arrivals():
    arr = serve.make_arrivals(rate=500.0, duration=20.0, mix=(0.6, 0.3, 0.1), ngraphs=8, seed=3)
    t = np.array([a[0] for a in arr])
    assert np.all(np.diff(t) > 0) and t[-1] < 20.0
    assert abs(len(arr) - 10000) < 4 * math.sqrt(10000)  # Poisson count around rate * duration
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 500.0) < 0.05 / 500.0 * 10
    kinds = [a[1] for a in arr]
    assert abs(kinds.count("bfs") / len(arr) - 0.6) < 0.03
    assert set(a[2] for a in arr) == set(range(8))
    assert arr == serve.make_arrivals(rate=500.0, duration=20.0, mix=(0.6, 0.3, 0.1), ngraphs=8, seed=3)


@pytest.mark.parametrize("max_large", [1, 3])
def test_two_queue_admission(max_large):
    # seven small graphs and one "large" one (the threshold is lowered to keep the graphs tiny)
    csrs = [gg.rmat(10, 16, seed=k + 1) for k in range(7)] + [gg.rmat(13, 16, seed=9)]
    large_n = 5000
    graphs = [FakeGraph(g.n) for g in csrs]
    fakes = []

    def factory(graphs, max_slots, budget, cfg):
        fakes.append(FakeServer(graphs, max_slots, large_n=large_n))
        return fakes[0]

    res = serve.serve(csrs, rate=400.0, duration=0.6, warmup=0.1, slice_ns=1, max_slots=16, budget_bytes=1 << 30,
                      cfg=Config(), graphs=graphs, drain_s=20.0, large_n=large_n, max_large=max_large,
                      server_factory=factory)
    f = fakes[0]
    assert 0 < f.max_large_seen <= max_large
    assert res["unfinished"] == 0 and res["completed"] == res["requests"]
    assert res["p50_ms"] is not None and res["p50_ms"] <= res["p99_ms"]
