"""The allocation-free BFS entry point (atos_bfs_noalloc) against the allocating one (atos_bfs).

atos_bfs_noalloc serves callers that cannot call cudaMalloc (an application whose own allocator
owns the device memory, a plug-in forbidden to allocate, a loop that cannot afford the device
synchronisation of an allocation): its scratch is a fixed array inside the library.  Two calls in
a row on the same GPU share that array, so the second call also checks that the first left nothing
behind.  The file sorts last so that a stop-at-first-failure run has already run every other test;
it needs nothing from the others and passes alone as well."""
import ctypes

import numpy as np
import pytest

import graphgen as gg
from gpu_common import atos_lib

pytestmark = pytest.mark.gpu

MAX_VERTICES = 262144  # ATOS_NOALLOC_MAX_VERTICES in include/atos.h


def _noalloc(L, rp, col, n, nnz, src, out, stream):
    return L.atos_bfs_noalloc(ctypes.c_void_p(rp), ctypes.c_void_p(col), n, nnz, src, ctypes.c_void_p(out),
                              ctypes.c_void_p(stream))


@pytest.mark.parametrize("maker,sources", [
    (lambda: gg.rmat(14, 16, seed=4), (0, 777)),
    (lambda: gg.grid(300, 211, delete_frac=0.1, seed=2), (0, 31000)),
])
def test_noalloc_matches_allocating_entry_point(maker, sources):
    atos = atos_lib()
    import torch
    g = maker()
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    L = atos.lib()
    with atos.Graph(rp, col) as G:
        for src in sources:  # two calls in a row on the shared scratch
            out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
            rc = _noalloc(L, rp.data_ptr(), col.data_ptr(), g.n, g.nnz, src, out.data_ptr(), stream)
            assert rc == 0, atos.status_string(rc)
            ref, st = G.bfs([src])
            assert st.status == 0
            assert torch.equal(out, ref[0]), f"source {src}: {(out != ref[0]).sum().item()} depths differ"


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
