"""Input generators: determinism, CSR well-formedness and exact sizes of the named workloads."""
import numpy as np
import pytest

import graphgen as gg


def assert_symmetric_simple_sorted(g):
    rp, col = g.row_ptr, g.col
    assert rp[0] == 0 and rp[-1] == g.nnz
    assert np.all(np.diff(rp) >= 0)
    assert col.size == 0 or (col.min() >= 0 and col.max() < g.n)
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rp))
    assert not np.any(src == col), "self-loop"
    for v in range(min(g.n, 2000)):
        row = col[rp[v]:rp[v + 1]]
        assert np.all(np.diff(row) > 0), f"row {v} not strictly increasing"
    a = set(zip(src.tolist(), col.tolist()))
    b = set(zip(col.tolist(), src.tolist()))
    assert a == b, "not symmetric"


@pytest.mark.parametrize("maker", [lambda: gg.rmat(8, seed=3), lambda: gg.grid(17, 9, delete_frac=0.1, seed=5),
                                   lambda: gg.rmat(9, seed=7, delete_frac=0.1)])
def test_csr_well_formed(maker):
    assert_symmetric_simple_sorted(maker())


def test_deterministic_and_seed_sensitive():
    a, b, c = gg.rmat(10, seed=11), gg.rmat(10, seed=11), gg.rmat(10, seed=12)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    assert not (a.nnz == c.nnz and np.array_equal(a.col, c.col))


def test_thread_count_invariant():
    a = gg.rmat(11, seed=4, delete_frac=0.1, nthreads=1)
    b = gg.rmat(11, seed=4, delete_frac=0.1, nthreads=5)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)


@pytest.mark.parametrize("w,h", [(64, 48), (5, 1), (1, 7), (33, 33)])
def test_grid_exact_edge_count(w, h):
    E = h * (w - 1) + (h - 1) * w
    g0 = gg.grid(w, h)
    assert g0.nnz == 2 * E
    g = gg.grid(w, h, delete_frac=0.1, seed=9)
    assert g.nnz == 2 * (E - int(0.1 * E))


def test_grid_2048_size():
    # 2048 x 2048 grid, 10% deletion: 8,384,512 edges, 838,451 deleted, 7,546,061 kept.
    g = gg.grid(2048, delete_frac=0.1, seed=1)
    assert g.n == 4194304 and g.nnz == 15092122


def test_grid_neighbours():
    g = gg.grid(4, 3)
    # vertex (1, 1) = 5 has neighbours 1, 4, 6, 9
    assert list(g.col[g.row_ptr[5]:g.row_ptr[6]]) == [1, 4, 6, 9]


def test_rmat_shape():
    g = gg.rmat(12, seed=1)
    assert g.n == 4096
    assert g.nnz == 96860  # regression value of the seeded generator
    deg = g.degrees
    # skew: vertex 0 is the hub (quadrant a = 0.57 is the top-left one, no permutation)
    assert deg[0] == deg.max()


def test_sources_have_degree():
    g = gg.rmat(10, seed=2)
    s = gg.sources(g, 64, seed=3)
    assert s.shape == (64,) and np.all(g.degrees[s] > 0)
    assert np.array_equal(s, gg.sources(g, 64, seed=3))


def test_from_edges_drops_loops_and_duplicates():
    g = gg.from_edges(4, [(0, 1), (1, 0), (2, 2), (1, 2), (1, 2)])
    assert list(g.row_ptr) == [0, 1, 3, 4, 4]
    assert list(g.col) == [1, 0, 2, 1]


def test_batched_mix_recipe():
    mix = gg.batched_mix()
    assert len(mix) == 256
    assert sum(1 for k, _, _ in mix if k == "rmat") == 128
    assert all(10 <= s <= 18 for k, s, _ in mix if k == "rmat")
    assert all(64 <= s <= 1024 for k, s, _ in mix if k == "grid")
    assert mix == gg.batched_mix()


def test_relabel_is_an_isomorphic_copy():
    g = gg.rmat(11, 8, seed=5)
    h, perm = gg.relabel(g, seed=3)
    assert np.array_equal(np.sort(perm), np.arange(g.n))  # a permutation
    assert not np.array_equal(perm, np.arange(g.n))
    assert h.n == g.n and h.nnz == g.nnz
    assert np.array_equal(h.degrees[perm], g.degrees)
    rows = np.repeat(np.arange(g.n), g.degrees)
    old = set(zip(perm[rows].tolist(), perm[g.col].tolist()))
    hrows = np.repeat(np.arange(h.n), h.degrees)
    assert old == set(zip(hrows.tolist(), h.col.tolist()))
    for v in range(h.n):  # rows sorted
        r = h.col[h.row_ptr[v]:h.row_ptr[v + 1]]
        assert np.all(np.diff(r) > 0)
    h2, perm2 = gg.relabel(g, seed=3, nthreads=1)  # the same for any thread count
    assert np.array_equal(perm, perm2) and np.array_equal(h.col, h2.col)
    assert not np.array_equal(perm, gg.relabel(g, seed=4)[1])
