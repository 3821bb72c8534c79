"""BFS on the GPU against the serial oracle: depths must be bit-exact (Section 5.1: the speculative
search reaches the exact hop distances whatever the pop order)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_common import thread_worker_configs, atos_lib, bfs_sources, configs, small_graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def atos():
    return atos_lib()


@pytest.fixture(scope="module")
def graphs():
    return small_graphs()


@pytest.mark.parametrize("gname", list(small_graphs().keys()))
def test_bfs_bit_exact_all_configs(atos, graphs, gname):
    g = graphs[gname]
    srcs = bfs_sources(g)
    refs = {s: oracle.bfs(g, s) for s in srcs}
    with atos.Graph.from_csr(g) as G:
        for cname, cfg in configs(atos).items():
            try:
                depths, st = G.bfs(srcs, cfg=cfg)
            except atos.AtosError as e:
                pytest.fail(f"{gname}/{cname}: {e}; queues {G.queue_state(len(srcs))}")
            d = depths.cpu().numpy()
            assert st.status == 0, (cname, st.status)
            for i, s in enumerate(srcs):
                bad = np.flatnonzero(d[i] != refs[s])
                assert bad.size == 0, f"{gname}/{cname} src {s}: {bad.size} depths differ, e.g. v{bad[0]} " \
                                      f"gpu {d[i][bad[0]]} oracle {refs[s][bad[0]]}"


def test_bfs_many_sources_windows(atos):
    g = gg.rmat(12, 16, seed=1)
    srcs = [int(x) for x in gg.sources(g, 40, seed=2)]
    refs = np.stack([oracle.bfs(g, s) for s in srcs])
    with atos.Graph.from_csr(g) as G:
        for window in (1, 3, 16, 40):
            for worker in (32, 256):
                cfg = atos.queue_config(window=window, worker_size=worker, fetch_size=32 if worker == 32 else 256)
                depths, st = G.bfs(srcs, cfg=cfg)
                assert st.status == 0
                assert np.array_equal(depths.cpu().numpy(), refs), (window, worker)


def test_bfs_stats_consistent(atos):
    g = gg.grid(64, 64, delete_frac=0.1, seed=1)
    ref = oracle.bfs(g, 0)
    reached = int((ref != oracle.UNREACHED).sum())
    with atos.Graph.from_csr(g) as G:
        _, st = G.bfs([0])
        # every reached vertex is popped at least once; every pop but the source's was a push
        assert st.tasks >= reached
        assert st.pushes == st.tasks - 1
        deg = g.degrees
        assert st.edges >= int(deg[ref != oracle.UNREACHED].sum())
        _, st = G.bfs([0], cfg=atos.queue_config("discrete-cta"))
        assert st.iterations == ref[ref != oracle.UNREACHED].max() + 1  # one generation per level
        assert st.tasks == reached  # level-synchronous: no overwork


def test_bfs_device_csr_borrow(atos):
    import torch
    g = gg.rmat(10, 16, seed=5)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    with atos.Graph(rp, col, borrow=True) as G:
        depths, _ = G.bfs([3])
        assert np.array_equal(depths.cpu().numpy()[0], oracle.bfs(g, 3))
    with atos.Graph(rp, col) as G:
        depths, _ = G.bfs([3])
        assert np.array_equal(depths.cpu().numpy()[0], oracle.bfs(g, 3))


def test_device_csr_validated(atos):
    """A CSR in device memory is checked before any kernel uses it: row_ptr on the host, every
    column index on the device, symmetry (when asked) on a host copy.  Out-of-range columns are
    only compared, never dereferenced."""
    import torch
    g = gg.rmat(10, 16, seed=5)
    rp = torch.from_numpy(g.row_ptr).cuda()
    for bad_value in (g.n, -1, 2**31 - 1):
        col = torch.from_numpy(g.col).cuda()
        col[g.nnz // 2] = bad_value
        for borrow in (False, True):
            with pytest.raises(atos.AtosError) as e:
                atos.Graph(rp, col, borrow=borrow)
            assert e.value.status == atos.abi.ERR_BAD_CSR, (bad_value, borrow)
    # a one-directional edge: accepted without the symmetry check, rejected with it
    one_way = gg.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    col = torch.from_numpy(one_way.col.copy()).cuda()
    col[0] = 2  # row 0 now holds (0, 2), whose mirror (2, 0) is missing
    rp1 = torch.from_numpy(one_way.row_ptr).cuda()
    with atos.Graph(rp1, col) as G:
        assert G.n == 4
    with pytest.raises(atos.AtosError) as e:
        atos.Graph(rp1, col, check_symmetric=True)
    assert e.value.status == atos.abi.ERR_BAD_CSR
    with atos.Graph(rp1, torch.from_numpy(one_way.col).cuda(), check_symmetric=True) as G:
        d, _ = G.bfs([0])
        assert np.array_equal(d.cpu().numpy()[0], oracle.bfs(one_way, 0))
    # a non-monotone row_ptr
    rp_bad = rp.clone()
    rp_bad[5] = rp_bad[7]
    with pytest.raises(atos.AtosError) as e:
        atos.Graph(rp_bad, torch.from_numpy(g.col).cuda())
    assert e.value.status == atos.abi.ERR_BAD_CSR


def test_bfs_invalid_arguments(atos):
    g = gg.path(10)
    with atos.Graph.from_csr(g) as G:
        for bad in ([10], [-1], []):
            with pytest.raises(atos.AtosError) as e:
                G.bfs(bad)
            assert e.value.status == atos.abi.ERR_INVALID_ARG
        with pytest.raises(atos.AtosError) as e:
            G.bfs([0], cfg=atos.queue_config(worker_size=96))
        assert e.value.status == atos.abi.ERR_UNSUPPORTED
        with pytest.raises(atos.AtosError) as e:
            G.bfs([0], cfg=atos.queue_config(worker_size=64, fetch_size=128))
        assert e.value.status == atos.abi.ERR_INVALID_ARG


def test_bfs_full_size_grid_2048(atos):
    """The 2048 x 2048 grid with 10% of edges deleted, BFS from the corner: bit-exact."""
    g = gg.grid(2048, delete_frac=0.1, seed=1)
    ref = oracle.bfs(g, 0)
    with atos.Graph.from_csr(g) as G:
        depths, st = G.bfs([0])
        assert st.status == 0
        assert np.array_equal(depths.cpu().numpy()[0], ref)


def test_bfs_full_size_rmat22_64_sources(atos):
    """RMAT scale 22, 64 seeded sources in one launch: four sampled sources bit-exact against the
    oracle, every source checked by the hop-distance certificate."""
    g = gg.rmat(22, 16, seed=1)
    srcs = [int(x) for x in gg.sources(g, 64, seed=1)]
    with atos.Graph.from_csr(g) as G:
        depths, st = G.bfs(srcs)
        assert st.status == 0
        d = depths.cpu().numpy()
    for i in (0, 21, 42, 63):
        assert np.array_equal(d[i], oracle.bfs(g, srcs[i])), f"source {srcs[i]}"
    for i in range(0, 64, 4):
        assert oracle.bfs_certificate(g, srcs[i], d[i]) == (0, -1), f"source {srcs[i]}"


@pytest.mark.parametrize("flags", ["host", "device_loop", "per_source", "per_source_device_loop", "groups_of_7",
                                   "groups_of_7_device_loop"])
def test_bfs_bsp_forms_many_sources(atos, flags):
    """The level-synchronous comparator (Algorithm 1) over 41 sources: the frontiers of all sources
    (or of groups of 7) in one launch per level, or one source after another, levels driven by the
    host or by a CUDA graph's conditional loop; bit-exact, with no overwork (each reached vertex
    expanded once per source) and one level per depth of each group."""
    f = {"host": 0, "device_loop": atos.FLAG_BSP_DEVICE_LOOP, "per_source": atos.FLAG_BSP_PER_SOURCE,
         "per_source_device_loop": atos.FLAG_BSP_PER_SOURCE | atos.FLAG_BSP_DEVICE_LOOP,
         "groups_of_7": 0, "groups_of_7_device_loop": atos.FLAG_BSP_DEVICE_LOOP}[flags]
    group = 1 if f & atos.FLAG_BSP_PER_SOURCE else (7 if "groups_of_7" in flags else 0)
    g = gg.rmat(12, 16, seed=1, delete_frac=0.1)
    srcs = [int(x) for x in gg.sources(g, 40, seed=2)] + [0]
    refs = np.stack([oracle.bfs(g, s) for s in srcs])
    reached = (refs != oracle.UNREACHED)
    ecc = np.where(reached, refs, 0).max(axis=1)
    with atos.Graph.from_csr(g) as G:
        for _ in range(2):  # a second run reuses the scratch (and the graph of the device loop)
            depths, st = G.bfs(srcs, cfg=atos.queue_config("bsp", flags=f, window=7 if group == 7 else 0))
            assert st.status == 0
            assert np.array_equal(depths.cpu().numpy(), refs)
            assert st.tasks == int(reached.sum())
            size = group or len(srcs)  # 4096 vertices: every source fits the default group
            levels = sum(int(ecc[i:i + size].max() + 1) for i in range(0, len(srcs), size))
            assert st.iterations == levels


def test_bfs_bsp_full_size(atos):
    """Full-size level-synchronous BFS: the 2048 x 2048 grid from the corner (thousands of
    levels, host-driven and in the device loop) bit-exact, and RMAT 22 with all 64 sources in one
    device-loop run (levels of more than 2^31 edges), sampled sources bit-exact and every fourth by
    the hop-distance certificate."""
    g = gg.grid(2048, delete_frac=0.1, seed=1)
    ref = oracle.bfs(g, 0)
    ecc = int(ref[ref != oracle.UNREACHED].max())
    with atos.Graph.from_csr(g) as G:
        for f in (0, atos.FLAG_BSP_DEVICE_LOOP):
            depths, st = G.bfs([0], cfg=atos.queue_config("bsp", flags=f))
            assert st.status == 0 and st.iterations == ecc + 1
            assert np.array_equal(depths.cpu().numpy()[0], ref)
    g = gg.rmat(22, 16, seed=1)
    srcs = [int(x) for x in gg.sources(g, 64, seed=1)]
    with atos.Graph.from_csr(g) as G:
        depths, st = G.bfs(srcs, cfg=atos.queue_config("bsp", flags=atos.FLAG_BSP_DEVICE_LOOP))
        assert st.status == 0
        d = depths.cpu().numpy()
    for i in (0, 37, 63):
        assert np.array_equal(d[i], oracle.bfs(g, srcs[i])), f"source {srcs[i]}"
    for i in range(0, 64, 4):
        assert oracle.bfs_certificate(g, srcs[i], d[i]) == (0, -1), f"source {srcs[i]}"


def test_bfs_expand_once_all_configs(atos):
    """ATOS_FLAG_BFS_EXPAND_ONCE: bit-exact depths for every configuration (BSP ignores the flag)."""
    for g in (gg.rmat(12, 16, seed=1), gg.grid(97, 61, delete_frac=0.1, seed=3), gg.rmat(11, 16, seed=7, delete_frac=0.1)):
        srcs = bfs_sources(g)
        ref = np.stack([oracle.bfs(g, s) for s in srcs])
        with atos.Graph.from_csr(g) as G:
            for cname, cfg in configs(atos).items():
                cfg.flags |= atos.FLAG_BFS_EXPAND_ONCE
                d, st = G.bfs(srcs, cfg=cfg)
                assert st.status == 0 and np.array_equal(d.cpu().numpy(), ref), cname


@pytest.mark.parametrize("gname", list(small_graphs().keys()))
def test_bfs_thread_workers_bit_exact(atos, graphs, gname):
    """Thread workers reach the same exact depths, with and without expansion markers."""
    g = graphs[gname]
    srcs = bfs_sources(g)
    ref = np.stack([oracle.bfs(g, s) for s in srcs])
    with atos.Graph.from_csr(g) as G:
        for cname, cfg in thread_worker_configs(atos).items():
            for marks in (False, True):
                if marks:
                    cfg.flags |= atos.FLAG_BFS_EXPAND_ONCE
                d, st = G.bfs(srcs, cfg=cfg)
                assert st.status == 0, (cname, marks, st.status)
                assert np.array_equal(d.cpu().numpy(), ref), (gname, cname, marks)
                assert st.tasks >= int((ref != oracle.UNREACHED).sum()), (cname, marks)


def test_bfs_thread_workers_windows_and_grid(atos):
    """Thread workers with instance windows over 40 sources, and on the 2048 x 2048 grid."""
    g = gg.rmat(12, 16, seed=1)
    srcs = [int(x) for x in gg.sources(g, 40, seed=2)]
    refs = np.stack([oracle.bfs(g, s) for s in srcs])
    with atos.Graph.from_csr(g) as G:
        for window in (1, 16):
            cfg = atos.queue_config(worker_size=1, fetch_size=32, window=window)
            d, st = G.bfs(srcs, cfg=cfg)
            assert st.status == 0 and np.array_equal(d.cpu().numpy(), refs), window
    g = gg.grid(2048, delete_frac=0.1, seed=1)
    ref = oracle.bfs(g, 0)
    with atos.Graph.from_csr(g) as G:
        d, st = G.bfs([0], cfg=atos.queue_config(worker_size=1, fetch_size=32))
        assert st.status == 0 and np.array_equal(d.cpu().numpy()[0], ref)


def test_thread_workers_arguments(atos):
    """A thread worker fetches at most 32 tasks (one per lane): a larger fetch size is an invalid
    argument, and the graph still works afterwards; servers pause CTA workers only."""
    g = gg.rmat(10, 8, seed=3)
    cfg = atos.queue_config(worker_size=1, fetch_size=32)
    with atos.Graph.from_csr(g) as G:
        with pytest.raises(atos.AtosError) as e:
            G.bfs([0], cfg=atos.queue_config(worker_size=1, fetch_size=64))
        assert e.value.status == atos.abi.ERR_INVALID_ARG
        d, st = G.bfs([0], cfg=cfg)
        assert np.array_equal(d.cpu().numpy()[0], oracle.bfs(g, 0))
        with pytest.raises(atos.AtosError) as e:
            atos.Server([G], max_slots=4, budget_bytes=1 << 26, cfg=cfg)
        assert e.value.status == atos.abi.ERR_UNSUPPORTED


def _hub_chain(k=3, leaves=12000, seed=4):
    """k hubs of `leaves` leaves each, hub i joined to hub i+1 by a path of i+2 edges and to a
    shared ring of 50 vertices, so the search reaches the hubs at several depths (and may reach a
    hub first by a longer route)."""
    pairs, nxt = [], 0
    hubs = list(range(k))
    nxt = k
    ring = list(range(nxt, nxt + 50))
    nxt += 50
    pairs += [(ring[i], ring[(i + 1) % 50]) for i in range(50)]
    for i, h in enumerate(hubs):
        pairs += [(h, nxt + j) for j in range(leaves)]
        nxt += leaves
        pairs.append((h, ring[(17 * i) % 50]))
        if i + 1 < k:
            path = list(range(nxt, nxt + i + 1))
            nxt += i + 1
            chain = [h] + path + [hubs[i + 1]]
            pairs += list(zip(chain[:-1], chain[1:]))
    return gg.from_edges(nxt, pairs, "hub_chain")


def test_bfs_split_rows(atos):
    """ATOS_FLAG_BFS_SPLIT_ROWS: rows longer than 8192 entries become segment tasks; depths stay
    bit-exact for every CTA configuration, with and without expansion markers, and more tasks
    are popped than vertices expanded (the segments).  Warp and thread workers ignore the flag."""
    for g in (gg.rmat(18, 16, seed=5), gg.star(20000), _hub_chain()):
        deg = np.diff(g.row_ptr)
        assert (deg > 8192).any()
        srcs = bfs_sources(g) + [int(np.argmax(deg))]
        ref = np.stack([oracle.bfs(g, s) for s in srcs])
        with atos.Graph.from_csr(g) as G:
            for cname, cfg in {**configs(atos), **thread_worker_configs(atos)}.items():
                if cname.startswith("bsp"):
                    continue
                base = cfg.flags | atos.FLAG_BFS_SPLIT_ROWS
                for extra in (0, atos.FLAG_BFS_EXPAND_ONCE):
                    cfg.flags = base | extra
                    d, st = G.bfs(srcs, cfg=cfg)
                    assert st.status == 0, (g.name, cname, extra, st.status)
                    assert np.array_equal(d.cpu().numpy(), ref), (g.name, cname, extra)
                    if cfg.worker_size > 32 and extra:
                        # the hub source's row alone is split into ceil(deg / 4096) segments
                        assert st.tasks > int((ref != oracle.UNREACHED).sum()), (g.name, cname)


def test_bfs_split_rows_many_sources(atos):
    """Segment tables of 64 sources run in windows of 8 and all at once (RMAT scale 18)."""
    g = gg.rmat(18, 16, seed=5)
    srcs = [int(x) for x in gg.sources(g, 64, seed=3)]
    refs = np.stack([oracle.bfs(g, s) for s in srcs[:8]])
    with atos.Graph.from_csr(g) as G:
        for window in (8, 0):
            cfg = atos.queue_config(worker_size=512, fetch_size=512, window=window,
                                    flags=atos.FLAG_BFS_SPLIT_ROWS | atos.FLAG_BFS_EXPAND_ONCE)
            d, st = G.bfs(srcs, cfg=cfg)
            assert st.status == 0
            d = d.cpu().numpy()
            assert np.array_equal(d[:8], refs), window
            for i in range(8, 64, 8):
                assert oracle.bfs_certificate(g, srcs[i], d[i]) == (0, -1), (window, srcs[i])
