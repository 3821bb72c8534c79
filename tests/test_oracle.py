"""Pins of the CPU oracle to facts it does not compute itself: closed forms, brute force,
library routines on small graphs, invariants, and planted mistakes that its checkers must catch.

Each group is chosen so that a plausible slip in oracle.c (a dropped term, a wrong sign, a
transposed operand, an off-by-one depth) fails at least one test here."""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle

UNR = oracle.UNREACHED
ALPHA = 0.85


def random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    return gg.from_edges(n, pairs, f"gnp{n}_{p}_{seed}")


def dense_adj(g):
    A = np.zeros((g.n, g.n))
    for v in range(g.n):
        A[v, g.col[g.row_ptr[v]:g.row_ptr[v + 1]]] = 1.0
    return A


# ----------------------------------------------------------------------------------- BFS pins

def floyd_warshall_hops(g):
    n = g.n
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0)
    A = dense_adj(g)
    D[A > 0] = 1
    for k in range(n):
        D = np.minimum(D, D[:, [k]] + D[[k], :])
    return D


def to_int_depth(row):
    return np.where(np.isinf(row), UNR, row).astype(np.int64)


def test_bfs_path_and_middle():
    g = gg.path(50)
    assert np.array_equal(oracle.bfs(g, 0), np.arange(50))
    assert np.array_equal(oracle.bfs(g, 20), np.abs(np.arange(50) - 20))


def test_bfs_grid_manhattan():
    w, h = 37, 23
    g = gg.grid(w, h)
    d = oracle.bfs(g, 0).reshape(h, w)
    r, c = np.mgrid[0:h, 0:w]
    assert np.array_equal(d, r + c)
    src = 11 * w + 7
    d = oracle.bfs(g, src).reshape(h, w)
    assert np.array_equal(d, np.abs(r - 11) + np.abs(c - 7))


def test_bfs_clique_star_disconnected():
    assert list(oracle.bfs(gg.clique(6), 2)) == [1, 1, 0, 1, 1, 1]
    assert list(oracle.bfs(gg.star(4), 3)) == [1, 2, 2, 0, 2]
    g = gg.from_edges(6, [(0, 1), (1, 2), (4, 5)])
    assert list(oracle.bfs(g, 0)) == [0, 1, 2, UNR, UNR, UNR]
    assert list(oracle.bfs(g, 3)) == [UNR, UNR, UNR, 0, UNR, UNR]


@pytest.mark.parametrize("seed", range(12))
def test_bfs_floyd_warshall(seed):
    n = 8 + 5 * seed
    g = random_graph(n, 0.08 + 0.02 * (seed % 4), seed)
    D = floyd_warshall_hops(g)
    for s in range(0, n, max(1, n // 6)):
        assert np.array_equal(oracle.bfs(g, s), to_int_depth(D[s]))


def test_bfs_scipy_shortest_path():
    sp = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sps
    g = gg.rmat(9, seed=5, delete_frac=0.1)
    M = sps.csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.n, g.n))
    for s in gg.sources(g, 5, seed=2):
        ref = sp.shortest_path(M, unweighted=True, indices=int(s))
        assert np.array_equal(oracle.bfs(g, s), to_int_depth(ref))


def test_bfs_certificate_accepts_and_rejects():
    g = gg.rmat(10, seed=3)
    d = oracle.bfs(g, 0)
    assert oracle.bfs_certificate(g, 0, d) == (0, -1)
    reached = np.flatnonzero((d != UNR) & (d > 0))
    unreached = np.flatnonzero(d == UNR)
    bad = d.copy(); bad[reached[5]] += 1                      # one depth too large
    assert oracle.bfs_certificate(g, 0, bad)[0] != 0
    bad = d.copy(); bad[reached[9]] -= 1                      # one depth too small
    assert oracle.bfs_certificate(g, 0, bad)[0] != 0
    bad = d.copy(); bad[reached[3]] = UNR                     # dropped vertex
    assert oracle.bfs_certificate(g, 0, bad)[0] == 2
    bad = d.copy(); bad[0] = 1                                # wrong source
    assert oracle.bfs_certificate(g, 0, bad)[0] == 1
    if unreached.size:
        bad = d.copy(); bad[unreached[0]] = 3                 # isolated vertex "reached"
        assert oracle.bfs_certificate(g, 0, bad)[0] != 0
    bad = d + 1; bad[d == UNR] = UNR; bad[0] = 0              # everything shifted
    assert oracle.bfs_certificate(g, 0, bad)[0] != 0


# ----------------------------------------------------------------------------- PageRank pins

def dense_fixed_point(g, alpha=ALPHA):
    """x = (1 - alpha)(I - alpha A D^-1)^-1 1, isolated vertices with zero column."""
    A = dense_adj(g)
    deg = A.sum(axis=0)
    P = np.divide(A, deg, out=np.zeros_like(A), where=deg > 0)
    return np.linalg.solve(np.eye(g.n) - alpha * P, (1 - alpha) * np.ones(g.n))


def test_pr_star_closed_form():
    for k in (1, 3, 10):
        x, _, _ = oracle.pagerank(gg.star(k), ALPHA)
        centre = (1 + ALPHA * k) / (1 + ALPHA)
        leaf = (1 - ALPHA) + ALPHA * centre / k
        assert x[0] == pytest.approx(centre, abs=1e-11)
        assert np.allclose(x[1:], leaf, atol=1e-11)
        assert x.sum() == pytest.approx(k + 1, abs=1e-10)


@pytest.mark.parametrize("g", [gg.cycle(17), gg.clique(9), gg.cycle(4)])
def test_pr_regular_graphs_uniform(g):
    x, _, _ = oracle.pagerank(g, ALPHA)
    assert np.allclose(x, 1.0, atol=1e-11)


@pytest.mark.parametrize("seed", range(6))
def test_pr_dense_solve(seed):
    g = random_graph(40 + 30 * seed, 0.05, seed)  # includes isolated vertices at low density
    x, _, _ = oracle.pagerank(g, ALPHA)
    ref = dense_fixed_point(g)
    assert np.abs(x - ref).sum() <= 1e-10 * g.n
    assert x.sum() == pytest.approx(oracle.fixed_point_sum(g, ALPHA), rel=1e-12)


def test_pr_alpha_dependence():
    g = random_graph(60, 0.1, 99)
    for a in (0.5, 0.85, 0.95):
        x, _, _ = oracle.pagerank(g, a)
        assert np.abs(x - dense_fixed_point(g, a)).sum() <= 1e-9 * g.n


def test_pr_networkx():
    nx = pytest.importorskip("networkx")
    g = gg.rmat(8, seed=2)
    keep = np.flatnonzero(g.degrees > 0)
    G = nx.Graph()
    G.add_nodes_from(keep.tolist())
    for v in keep:
        for w in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]:
            G.add_edge(int(v), int(w))
    ref = nx.pagerank(G, alpha=ALPHA, tol=1e-15, max_iter=10000)
    x, _, _ = oracle.pagerank(g, ALPHA)
    xs = x[keep] / x[keep].sum()
    r = np.array([ref[int(v)] for v in keep])
    assert np.abs(xs - r).sum() < 1e-9


def test_pr_residual_bound_holds_and_detects():
    g = random_graph(120, 0.04, 7)
    p = dense_fixed_point(g)
    q0 = p / p.sum()
    assert oracle.pr_error_bound(g, q0) < 1e-12
    rng = np.random.default_rng(0)
    for scale in (1e-6, 1e-4, 1e-2):
        q = q0 * (1 + scale * rng.standard_normal(g.n))
        q = np.abs(q) / np.abs(q).sum()
        true = np.abs(q - q0).sum()
        bound = oracle.pr_error_bound(g, q)
        assert bound >= true * (1 - 1e-9)
        assert bound > 0.1 * true  # not vacuous either


def test_pr_push_serial_invariant_and_epsilon():
    """Algorithm 3's steps serially: the invariant p = rank + (I - alpha P)^-1 residue pins the
    reading of the initial residue, and every residue ends at or below epsilon."""
    g = random_graph(90, 0.06, 3)
    eps = 1e-9
    rank, res, pushes, ep = oracle.pr_push_serial(g, ALPHA, eps)
    A = dense_adj(g)
    deg = A.sum(axis=0)
    P = np.divide(A, deg, out=np.zeros_like(A), where=deg > 0)
    p = dense_fixed_point(g)
    assert np.abs(rank + np.linalg.solve(np.eye(g.n) - ALPHA * P, res) - p).max() < 1e-12
    assert res.max() <= eps
    assert np.abs(rank - p).sum() <= res.sum() / (1 - ALPHA) + 1e-12
    assert pushes > 0 and ep >= pushes


def test_pr_push_serial_matches_power_iteration():
    g = gg.rmat(10, seed=4)
    x, _, _ = oracle.pagerank(g, ALPHA)
    rank, res, _, _ = oracle.pr_push_serial(g, ALPHA, 1e-9)
    assert np.abs(rank / rank.sum() - x / x.sum()).sum() < 1e-7


# ----------------------------------------------------------------------------- colouring pins

def chromatic_number(g):
    for k in range(1, g.n + 1):
        for col in itertools.product(range(k), repeat=g.n):
            if all(col[v] != col[w] for v in range(g.n) for w in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]):
                return k
    return g.n


def test_greedy_grid_two_colours():
    w, h = 13, 7
    c, k = oracle.greedy_color(gg.grid(w, h))
    r, cc = np.mgrid[0:h, 0:w]
    assert k == 2 and np.array_equal(c.reshape(h, w), (r + cc) % 2)


@pytest.mark.parametrize("g,k", [(gg.clique(7), 7), (gg.cycle(9), 3), (gg.cycle(10), 2), (gg.star(6), 2),
                                 (gg.path(8), 2)])
def test_greedy_known_counts(g, k):
    c, kk = oracle.greedy_color(g)
    assert kk == k
    assert oracle.check_coloring(g, c)[0] == 0


@pytest.mark.parametrize("seed", range(5))
def test_greedy_vs_exhaustive_chromatic(seed):
    g = random_graph(8, 0.45, seed)
    c, k = oracle.greedy_color(g)
    assert oracle.check_coloring(g, c)[0] == 0
    assert k >= chromatic_number(g)


def test_greedy_networkx_same_order():
    nx = pytest.importorskip("networkx")
    g = gg.rmat(9, seed=8)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for v in range(g.n):
        for w in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]:
            G.add_edge(v, int(w))
    ref = nx.greedy_color(G, strategy=lambda G_, colors: list(range(g.n)))
    c, _ = oracle.greedy_color(g)
    assert all(c[v] == ref[v] for v in range(g.n))
    order = np.random.default_rng(1).permutation(g.n).astype(np.int32)
    ref = nx.greedy_color(G, strategy=lambda G_, colors: [int(v) for v in order])
    c, _ = oracle.greedy_color(g, order)
    assert all(c[v] == ref[v] for v in range(g.n))


def test_greedy_first_fit_range():
    g = gg.rmat(11, seed=2)
    c, k = oracle.greedy_color(g)
    assert np.all(c <= g.degrees) and np.all(c >= 0)


def test_check_coloring_rejects_planted_mistakes():
    g = gg.rmat(9, seed=6)
    c, _ = oracle.greedy_color(g)
    v = int(np.argmax(g.degrees))
    w = int(g.col[g.row_ptr[v]])
    bad = c.copy(); bad[w] = bad[v]
    assert oracle.check_coloring(g, bad)[0] == 1
    bad = c.copy(); bad[v] = g.degrees[v] + 1
    assert oracle.check_coloring(g, bad)[0] in (1, 2)
    iso = np.flatnonzero(g.degrees == 0)
    if iso.size:
        bad = c.copy(); bad[iso[0]] = 1
        assert oracle.check_coloring(g, bad)[0] == 2
    bad = c.copy(); bad[3] = -1
    assert oracle.check_coloring(g, bad)[0] == 3


# ------------------------------------------------------------------- stored oracle regressions

@pytest.mark.parametrize("fname,maker", [
    ("rmat12_s1.json", lambda: gg.rmat(12, 16, seed=1)),
    ("grid64_del10_s1.json", lambda: gg.grid(64, 64, delete_frac=0.1, seed=1)),
])
def test_golden_regression(fname, maker):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", fname)) as f:
        ref = json.load(f)
    g = maker()
    assert (g.n, g.nnz) == (ref["n"], ref["nnz"])
    for s, info in ref["bfs"].items():
        d = oracle.bfs(g, int(s))
        r = d[d != UNR]
        assert r.size == info["reached"]
        assert np.bincount(r).tolist() == info["depth_histogram"]
    x, _, _ = oracle.pagerank(g, 0.85)
    assert x.sum() == pytest.approx(ref["pagerank"]["sum_unnormalised"], rel=1e-12)
    q = x / x.sum()
    for v, val in ref["pagerank"]["top"]:
        assert q[v] == pytest.approx(val, rel=1e-10)
    assert oracle.greedy_color(g)[1] == ref["greedy_colors"]


def test_pr_rounding_floor_stop():
    """On a large star the FP64 step cannot fall below 1e-13 per vertex (the centre holds ~n/2);
    the iteration must still stop, at the rounding floor, with the closed-form values."""
    k = 1000
    x, sweeps, last = oracle.pagerank(gg.star(k), ALPHA)
    centre = (1 + ALPHA * k) / (1 + ALPHA)
    assert x[0] == pytest.approx(centre, rel=1e-12)
    assert np.allclose(x[1:], (1 - ALPHA) + ALPHA * centre / k, rtol=1e-12)


def test_relabelling_invariance():
    """Renaming the vertices renames the results: BFS depths and the PageRank fixed point follow
    the permutation; greedy colouring in the renamed order is still proper and equals greedy on the
    original graph in the order perm^-1 (first fit depends only on the visiting order)."""
    g = gg.rmat(10, 8, seed=9)
    h, perm = gg.relabel(g, seed=2)
    s = int(gg.sources(g, 1, seed=4)[0])
    assert np.array_equal(oracle.bfs(h, int(perm[s]))[perm], oracle.bfs(g, s))
    assert np.allclose(oracle.pagerank(h)[0][perm], oracle.pagerank(g)[0], rtol=0, atol=1e-10)
    ch, kh = oracle.greedy_color(h)
    assert oracle.check_coloring(h, ch)[0] == 0
    inv = np.argsort(perm)  # vertex of g visited at step i of h's id order
    cg, kg = oracle.greedy_color(g, order=inv)
    assert kg == kh and np.array_equal(ch[perm], cg)
