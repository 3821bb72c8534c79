"""The allocation-free BFS entry point (atos_bfs_noalloc) against the CPU oracle and the
allocating entry point (atos_bfs).

atos_bfs_noalloc serves callers that cannot call cudaMalloc (an application whose own allocator
owns the device memory, a plug-in forbidden to allocate, a loop that cannot afford the device
synchronisation of an allocation): its scratch is a fixed array inside the library.  Calls in a
row on the same GPU share that array, so every later call also checks that the earlier ones
(smaller graphs, larger graphs, a rejected malformed graph) left nothing behind.  The file sorts
last so that a stop-at-first-failure run has already run every other test; it needs nothing from
the others and passes alone as well."""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_common import atos_lib

pytestmark = pytest.mark.gpu

MAX_VERTICES = 262144  # ATOS_NOALLOC_MAX_VERTICES in include/atos.h


def _noalloc(L, rp, col, n, nnz, src, out, stream):
    return L.atos_bfs_noalloc(ctypes.c_void_p(rp), ctypes.c_void_p(col), n, nnz, src, ctypes.c_void_p(out),
                              ctypes.c_void_p(stream))


def _run(atos, g, src):
    """One call on g from src; returns the depths on the host."""
    import torch
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col if g.nnz else np.zeros(1, np.int32)).cuda()
    out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = _noalloc(atos.lib(), rp.data_ptr(), col.data_ptr(), g.n, g.nnz, src, out.data_ptr(), stream)
    assert rc == 0, atos.status_string(rc)
    return out.cpu().numpy()


@pytest.mark.parametrize("maker,sources", [
    (lambda: gg.rmat(14, 16, seed=4), (0, 777)),
    (lambda: gg.grid(300, 211, delete_frac=0.1, seed=2), (0, 31000)),
])
def test_noalloc_matches_oracle_and_allocating_entry_point(maker, sources):
    atos = atos_lib()
    import torch
    g = maker()
    with atos.Graph(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda()) as G:
        for src in sources:  # two calls in a row on the shared scratch
            got = _run(atos, g, src)
            assert np.array_equal(got, oracle.bfs(g, src)), f"source {src}: depths differ from the oracle"
            ref, st = G.bfs([src])
            assert st.status == 0
            assert np.array_equal(got, ref[0].cpu().numpy()), f"source {src}: differs from atos_bfs"


def test_noalloc_at_its_size_limit_after_a_small_graph():
    """Graphs of exactly ATOS_NOALLOC_MAX_VERTICES vertices (a mesh and a scale-free graph), each
    after a call on a small graph, so the shared ring is reused across sizes."""
    atos = atos_lib()
    small = gg.path(50)
    for big in (gg.grid(512, 512, delete_frac=0.1, seed=5), gg.rmat(18, 16, seed=6)):
        assert big.n == MAX_VERTICES
        assert np.array_equal(_run(atos, small, 7), oracle.bfs(small, 7))
        src = int(gg.sources(big, 1, seed=9)[0])
        for s in (0, src):
            assert np.array_equal(_run(atos, big, s), oracle.bfs(big, s)), f"{big.name} from {s}"


def test_noalloc_rejects_malformed_csr_before_the_search():
    """Each CSR below breaks one rule; the device check rejects it and the search never reads it.
    A valid call right after shows the shared scratch is still usable."""
    atos = atos_lib()
    import torch
    L = atos.lib()
    stream = torch.cuda.current_stream().cuda_stream
    g = gg.grid(20, 20, seed=1)
    bad_cases = {}
    col = g.col.copy()
    col[17] = g.n  # a column index out of range
    bad_cases["col_out_of_range"] = (g.row_ptr, col, g.nnz)
    col = g.col.copy()
    col[3] = -1
    bad_cases["negative_col"] = (g.row_ptr, col, g.nnz)
    rp = g.row_ptr.copy()
    rp[5], rp[6] = rp[6], rp[5]  # a row that ends before it starts
    bad_cases["rows_decrease"] = (rp, g.col, g.nnz)
    bad_cases["nnz_mismatch"] = (g.row_ptr, g.col, g.nnz - 1)
    rp = g.row_ptr.copy()
    rp[0] = 1
    bad_cases["first_row_ptr"] = (rp, g.col, g.nnz)
    for name, (rp_h, col_h, nnz) in bad_cases.items():
        rp_d = torch.from_numpy(np.ascontiguousarray(rp_h)).cuda()
        col_d = torch.from_numpy(np.ascontiguousarray(col_h)).cuda()
        out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        rc = _noalloc(L, rp_d.data_ptr(), col_d.data_ptr(), g.n, nnz, 0, out.data_ptr(), stream)
        assert rc == atos.abi.ERR_BAD_CSR, f"{name}: {atos.status_string(rc)}"
        assert bool((out == -7).all()), f"{name}: the output was written"
    assert np.array_equal(_run(atos, g, 0), oracle.bfs(g, 0))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    atos = atos_lib()
    import torch
    L = atos.lib()
    stream = torch.cuda.current_stream().cuda_stream
    rp = torch.zeros(MAX_VERTICES + 2, dtype=torch.int32, device="cuda")
    out = torch.empty(MAX_VERTICES + 1, dtype=torch.int32, device="cuda")
    rc = _noalloc(L, rp.data_ptr(), rp.data_ptr(), MAX_VERTICES + 1, 0, 0, out.data_ptr(), stream)
    assert rc == atos.abi.ERR_INVALID_ARG
    rc = _noalloc(L, rp.data_ptr(), rp.data_ptr(), MAX_VERTICES, 0, MAX_VERTICES, out.data_ptr(), stream)
    assert rc == atos.abi.ERR_INVALID_ARG  # source out of range
