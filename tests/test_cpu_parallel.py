"""The multi-threaded CPU baseline against the serial oracle: exact BFS depths, the PageRank
fixed point within its stopping tolerance, proper colourings."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import parallel


@pytest.mark.parametrize("nthreads", [1, 4])
def test_parallel_bfs_exact(nthreads):
    for g in (gg.rmat(12, 16, seed=1), gg.grid(61, 47, delete_frac=0.1, seed=2), gg.path(50)):
        srcs = gg.sources(g, 6, seed=3)
        for s in (srcs[:2], srcs):  # fewer sources than threads: level-parallel; more: one per thread
            d, edges = parallel.bfs(g, s, nthreads=nthreads)
            for i, s0 in enumerate(s):
                assert np.array_equal(d[i], oracle.bfs(g, int(s0)))
            reached = sum(int(g.degrees[d[i] != oracle.UNREACHED].sum()) for i in range(len(s)))
            assert edges == reached  # every reached vertex's row read once


@pytest.mark.parametrize("nthreads", [1, 4])
def test_parallel_pagerank_fixed_point(nthreads):
    g = gg.rmat(11, 8, seed=4)
    x, it = parallel.pagerank(g, 0.85, 1e-12, nthreads=nthreads)
    ref = oracle.pagerank(g)[0]
    assert it > 10
    # a sweep whose L1 change is delta leaves at most alpha / (1 - alpha) * delta to the fixed point
    assert np.abs(x - ref).sum() <= 0.85 / 0.15 * 1e-12 * g.n * 1.01 + 1e-9
    assert oracle.pr_error_bound(g, x / x.sum()) < 1e-9


@pytest.mark.parametrize("nthreads", [1, 4])
def test_parallel_color_proper(nthreads):
    for g in (gg.rmat(12, 16, seed=1), gg.grid(64, 64), gg.clique(30), gg.cycle(9)):
        c, k, rounds, edges = parallel.color(g, nthreads=nthreads)
        code, _, used = oracle.check_coloring(g, c)
        assert code == 0 and used == k and rounds >= 1 and edges >= 2 * g.nnz
    for g in (gg.clique(30), gg.rmat(10, 8, seed=2)):  # one thread, id order: exactly serial greedy
        c, k, rounds, _ = parallel.color(g, nthreads=1)
        ref, kref = oracle.greedy_color(g)
        assert rounds == 1 and k == kref and np.array_equal(c, ref)
