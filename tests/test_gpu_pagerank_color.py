"""PageRank and colouring on the GPU against the oracle.

PageRank (Section 5.2): the normalised FP32 result must be within L1 1e-4 of the FP64 fixed point,
and the FP64 error bound the library reports must cover the actual distance.  Colouring
(Section 5.3): several colourings are correct, so the test checks what is unique -- properness and
the first-fit range 0 <= c(v) <= deg(v) -- and reports the colour count next to serial greedy."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_common import ALPHA, EPS, PR_L1_TOL, atos_lib, configs, small_graphs, thread_worker_configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def atos():
    return atos_lib()


@pytest.fixture(scope="module")
def graphs():
    return small_graphs()


def pr_reference(g):
    x, _, _ = oracle.pagerank(g, ALPHA)
    return x / x.sum()


@pytest.mark.parametrize("gname", ["rmat12", "rmat11_del", "grid97x61_del", "star1000", "clique40", "two_parts",
                                   "path300", "single", "isolated3"])
def test_pagerank_all_configs(atos, graphs, gname):
    g = graphs[gname]
    ref = pr_reference(g)
    with atos.Graph.from_csr(g) as G:
        for cname, cfg in configs(atos).items():
            try:
                rank, st = G.pagerank(ALPHA, EPS, cfg=cfg)
            except atos.AtosError as e:
                pytest.fail(f"{gname}/{cname}: {e}; queues {G.queue_state(1)}")
            assert st.status == 0, cname
            q = rank.cpu().numpy().astype(np.float64)
            l1 = np.abs(q - ref).sum()
            assert l1 <= PR_L1_TOL, f"{gname}/{cname}: L1 {l1}"
            assert abs(q.sum() - 1.0) < 1e-5
            assert st.error_bound <= PR_L1_TOL, f"{gname}/{cname}: bound {st.error_bound}"
            assert l1 <= st.error_bound * 1.0001 + 1e-12, f"{gname}/{cname}: L1 {l1} > bound {st.error_bound}"


def test_pagerank_check_size_and_epsilon(atos):
    g = gg.rmat(12, 16, seed=1)
    ref = pr_reference(g)
    with atos.Graph.from_csr(g) as G:
        for cs in (1, 8, 128):
            rank, st = G.pagerank(ALPHA, EPS, cfg=atos.queue_config(check_size=cs))
            assert np.abs(rank.cpu().numpy() - ref).sum() <= PR_L1_TOL
        # a loose epsilon still meets its own bound and does less work
        _, tight = G.pagerank(ALPHA, 1e-9)
        rank, loose = G.pagerank(ALPHA, 1e-5)
        assert loose.edges < tight.edges
        l1 = np.abs(rank.cpu().numpy() - ref).sum()
        assert l1 <= loose.error_bound * 1.0001


def test_pagerank_invalid(atos):
    with atos.Graph.from_csr(gg.path(5)) as G:
        for a in (0.0, 1.0, -0.5):
            with pytest.raises(atos.AtosError):
                G.pagerank(a, EPS)
        with pytest.raises(atos.AtosError):
            G.pagerank(ALPHA, 0.0)


def test_pagerank_full_size_grid_2048(atos):
    """FP32 push PageRank on the 2048^2 grid (10% deletion), eps 1e-9, against the FP64 oracle."""
    g = gg.grid(2048, delete_frac=0.1, seed=1)
    ref = pr_reference(g)
    with atos.Graph.from_csr(g) as G:
        rank, st = G.pagerank(ALPHA, EPS)
    q = rank.cpu().numpy().astype(np.float64)
    l1 = np.abs(q - ref).sum()
    assert st.status == 0 and l1 <= PR_L1_TOL and l1 <= st.error_bound * 1.0001
    # the CPU certificate agrees with the bound the library computed on the device
    assert oracle.pr_error_bound(g, q / q.sum(), ALPHA) <= PR_L1_TOL


@pytest.mark.parametrize("gname", list(small_graphs().keys()))
def test_color_proper_all_configs(atos, graphs, gname):
    g = graphs[gname]
    _, greedy = oracle.greedy_color(g)
    with atos.Graph.from_csr(g) as G:
        for cname, cfg in configs(atos).items():
            try:
                colors, k, st = G.color(cfg=cfg)
            except atos.AtosError as e:
                pytest.fail(f"{gname}/{cname}: {e}; queues {G.queue_state(1)}")
            assert st.status == 0, cname
            c = colors.cpu().numpy()
            code, bad, kk = oracle.check_coloring(g, c)
            assert code == 0, f"{gname}/{cname}: code {code} at vertex {bad}"
            assert k == kk == st.num_colors
            # first fit never needs more than max degree + 1 colours
            assert k <= int(g.degrees.max()) + 1


def test_color_known_graphs(atos):
    with atos.Graph.from_csr(gg.clique(17)) as G:
        _, k, _ = G.color()
        assert k == 17
    with atos.Graph.from_csr(gg.grid(40, 30)) as G:
        colors, k, _ = G.color()
        assert 2 <= k <= 5 and oracle.check_coloring(gg.grid(40, 30), colors.cpu().numpy())[0] == 0
    with atos.Graph.from_csr(gg.star(300)) as G:
        _, k, _ = G.color()
        assert k == 2


def test_color_full_size_rmat22(atos):
    g = gg.rmat(22, 16, seed=1)
    _, greedy = oracle.greedy_color(g)
    with atos.Graph.from_csr(g) as G:
        colors, k, st = G.color()
    code, bad, kk = oracle.check_coloring(g, colors.cpu().numpy())
    assert st.status == 0 and code == 0 and k == kk
    print(f"rmat22 colouring: {k} colours (serial greedy {greedy}), {st.tasks / g.n:.3f} tasks per vertex")


@pytest.mark.parametrize("worker", [256, 1024])
def test_pagerank_full_size_rmat22_certificate(atos, worker):
    """RMAT 22 is too large for the FP64 power iteration in a test; the FP64 residual certificate
    (computed on the CPU from the GPU result) bounds the distance to the fixed point instead."""
    g = gg.rmat(22, 16, seed=1)
    flags = 0
    with atos.Graph.from_csr(g) as G:
        rank, st = G.pagerank(ALPHA, EPS, cfg=atos.queue_config(worker_size=worker, fetch_size=worker))
    q = rank.cpu().numpy().astype(np.float64)
    bound = oracle.pr_error_bound(g, q / q.sum(), ALPHA)
    assert st.status == 0 and bound <= PR_L1_TOL and st.error_bound <= PR_L1_TOL
    print(f"rmat22 pagerank flags {flags}: bound {bound:.3e} (device {st.error_bound:.3e}), {st.tasks} tasks, "
          f"{st.edges} edge pushes, {st.ms:.1f} ms")


@pytest.mark.parametrize("worker", [1024, 512, 32])
def test_repeated_runs_leave_scratch_clean(atos, worker):
    """Every successful run must leave no queued bit set and no ring slot occupied, or the next
    run on the same graph object could take a stale item (a race in the final PageRank sweep
    once left items pushed after termination)."""
    g = gg.clique(40)
    ref = pr_reference(g)
    cfg = atos.queue_config(worker_size=worker, fetch_size=32 if worker == 32 else worker)
    with atos.Graph.from_csr(g) as G:
        for rep in range(12):
            rank, st = G.pagerank(ALPHA, EPS, cfg=cfg)
            assert np.abs(rank.cpu().numpy() - ref).sum() <= PR_L1_TOL, f"rep {rep}"
            assert G.scratch_check() == (0, 0), f"rep {rep}: {G.scratch_check()}"
            colors, k, _ = G.color(cfg=cfg)
            assert k == 40 and G.scratch_check() == (0, 0)
            G.bfs([rep % 40], cfg=cfg)
            assert G.scratch_check()[1] == 0


@pytest.mark.parametrize("gname", ["rmat12", "rmat11_del", "grid97x61_del", "star1000", "clique40", "two_parts",
                                   "path300", "single", "isolated3"])
def test_pagerank_crossing_all_configs(atos, graphs, gname):
    """Threshold-crossing enqueue (ATOS_FLAG_PR_CROSSING): the same fixed point, tolerance and
    bound as Algorithm 4's Check_Size scan, for every worker shape and strategy."""
    g = graphs[gname]
    ref = pr_reference(g)
    with atos.Graph.from_csr(g) as G:
        for cname, cfg in configs(atos).items():
            cfg.flags |= atos.FLAG_PR_CROSSING
            try:
                rank, st = G.pagerank(ALPHA, EPS, cfg=cfg)
            except atos.AtosError as e:
                pytest.fail(f"{gname}/{cname}: {e}; queues {G.queue_state(1)}")
            q = rank.cpu().numpy().astype(np.float64)
            l1 = np.abs(q - ref).sum()
            assert st.status == 0 and l1 <= PR_L1_TOL, f"{gname}/{cname}: L1 {l1}"
            assert l1 <= st.error_bound * 1.0001 + 1e-12, f"{gname}/{cname}: L1 {l1} > bound {st.error_bound}"
            if not cname.startswith("bsp"):  # the level-synchronous form uses neither the ring nor the queued bits
                assert G.scratch_check() == (0, 0), f"{gname}/{cname}: {G.scratch_check()}"


def test_pagerank_crossing_full_size_grid_2048(atos):
    """The crossing rule on the high-diameter mesh (where it beats the Check_Size scan); on
    RMAT graphs it multiplies the work and its FP32 rank sums lose small residues, which is why
    the autotuner gates PageRank candidates on their error bound."""
    g = gg.grid(2048, delete_frac=0.1, seed=1)
    ref = pr_reference(g)
    with atos.Graph.from_csr(g) as G:
        for worker in (256, 1024):
            cfg = atos.queue_config(worker_size=worker, fetch_size=worker, flags=atos.FLAG_PR_CROSSING)
            rank, st = G.pagerank(ALPHA, EPS, cfg=cfg)
            l1 = np.abs(rank.cpu().numpy().astype(np.float64) - ref).sum()
            assert st.status == 0 and l1 <= PR_L1_TOL and l1 <= st.error_bound * 1.0001, f"cta{worker}: L1 {l1}"


def test_unknown_config_flag_rejected(atos):
    with atos.Graph.from_csr(gg.path(5)) as G:
        with pytest.raises(atos.AtosError) as e:
            G.pagerank(ALPHA, EPS, cfg=atos.queue_config(flags=1 << 20))
        assert e.value.status == atos.abi.ERR_INVALID_ARG


def test_stats_batches_and_idle_polls(atos):
    """tasks / batches is the mean worker batch; persistent CTA workers never run more tasks per
    batch than their fetch size."""
    g = gg.rmat(12, 16, seed=1)
    with atos.Graph.from_csr(g) as G:
        for worker, fetch in ((256, 256), (1024, 1024), (128, 16), (32, 32)):
            _, st = G.pagerank(ALPHA, EPS, cfg=atos.queue_config(worker_size=worker, fetch_size=fetch))
            assert st.batches > 0 and st.tasks <= st.batches * fetch, (worker, st.as_dict())
            _, st = G.bfs([0], cfg=atos.queue_config(worker_size=worker, fetch_size=fetch))
            assert 0 < st.batches <= st.tasks <= st.batches * fetch
        _, st = G.pagerank(ALPHA, EPS, cfg=atos.queue_config("bsp"))
        assert st.batches == 0


@pytest.mark.parametrize("gname", ["rmat12", "rmat11_del", "grid97x61_del", "star1000", "clique40", "two_parts",
                                   "path300", "single", "isolated3"])
def test_spread_ids_all_configs(atos, graphs, gname):
    """PageRank and colouring on the spread-id copy of the graph (ATOS_FLAG_SPREAD_IDS): results in
    the caller's ids, the same gates as on the original layout."""
    g = graphs[gname]
    ref = pr_reference(g)
    with atos.Graph.from_csr(g) as G:
        for cname, cfg in configs(atos).items():
            cfg.flags |= atos.FLAG_SPREAD_IDS
            rank, st = G.pagerank(ALPHA, EPS, cfg=cfg)
            q = rank.cpu().numpy().astype(np.float64)
            l1 = np.abs(q - ref).sum()
            assert st.status == 0 and l1 <= PR_L1_TOL, f"{gname}/{cname}: L1 {l1}"
            assert l1 <= st.error_bound * 1.0001 + 1e-12, f"{gname}/{cname}: L1 {l1} > bound {st.error_bound}"
            colors, k, st = G.color(cfg=cfg)
            code, bad, kk = oracle.check_coloring(g, colors.cpu().numpy())
            assert st.status == 0 and code == 0 and k == kk, f"{gname}/{cname}: code {code} vertex {bad}"
            if not cname.startswith("bsp"):
                assert G.scratch_check() == (0, 0), f"{gname}/{cname}: {G.scratch_check()}"


def _degree_class(d):
    """Four classes per power of two: 0 for isolated vertices, else 1 + 4 floor(log2 d) + the two
    bits below d's leading one."""
    if d <= 0:
        return 0
    lg = int(d).bit_length() - 1
    sub = (d >> (lg - 2)) & 3 if lg >= 2 else (d << (2 - lg)) & 3
    return 1 + 4 * lg + sub


@pytest.mark.parametrize("maker", [lambda: gg.rmat(12, 16, seed=1), lambda: gg.rmat(16, 16, seed=2),
                                   lambda: gg.rmat(11, 16, seed=7, delete_frac=0.1),
                                   lambda: gg.grid(97, 61, delete_frac=0.1, seed=3), lambda: gg.star(1000),
                                   lambda: gg.from_edges(70, [(0, 1)], "edge_and_isolated")])
def test_spread_layout_hub_region(atos, maker):
    """The spread-id copy's layout: a bijection; the H hubs are the largest degree classes, whole,
    as many as fit in min(16384, 2^k) (2^k the largest power of two <= n / 32), and the hub of
    rank i (largest class first, ids increasing within a class) has the id 32 ((mul i + add) mod
    2^k) for one odd mul: at most one hub per 128-byte line."""
    g = maker()
    with atos.Graph.from_csr(g) as G:
        perm, H = G.spread_layout()
    assert np.array_equal(np.sort(perm), np.arange(g.n)), "not a permutation"
    lines = 0
    if g.n >= 32:
        lines = 1
        while lines * 2 <= g.n // 32:
            lines *= 2
    cap = min(16384, lines)
    assert 0 <= H <= cap
    cls = np.array([_degree_class(int(d)) for d in g.degrees])
    # the hubs by rank, from the degree classes alone
    order = sorted((v for v in range(g.n) if cls[v] > 0), key=lambda v: (-cls[v], v))
    hv = np.array(order[:H], dtype=np.int64)
    if H:
        bmin = cls[hv].min()
        assert H == np.count_nonzero(cls >= bmin), "hubs are not whole degree classes"
    rest = cls[(cls > 0)]
    if H < rest.size:  # the next class down did not fit
        nxt = cls[order[H]]
        assert H + np.count_nonzero(cls == nxt) > cap
    ids = perm[hv]
    assert np.all(ids % 32 == 0) and np.all(ids < 32 * max(lines, 1))
    if H >= 2:
        add = ids[0] // 32
        mul = (ids[1] // 32 - add) % lines
        assert mul % 2 == 1
        want = 32 * ((mul * np.arange(H, dtype=np.int64) + add) % lines)
        assert np.array_equal(ids, want), "hub ids do not follow one odd multiplier"
    # no other vertex shares a line with a hub at its first entry
    assert len(set((ids // 32).tolist())) == H


@pytest.mark.parametrize("worker", [64, 256, 512, 1024])
def test_pagerank_hub_combining_rmat16(atos, worker):
    """RMAT 16 on the spread layout: its hubs (up to 2048) outnumber the shared-memory accumulators
    of the 64-thread CTA worker and fit those of the larger ones; the result matches the oracle
    either way."""
    g = gg.rmat(16, 16, seed=2)
    ref = pr_reference(g)
    cfg = atos.queue_config(worker_size=worker, fetch_size=worker, check_size=8, flags=atos.FLAG_SPREAD_IDS)
    with atos.Graph.from_csr(g) as G:
        _, H = G.spread_layout()
        assert H > 512
        rank, st = G.pagerank(ALPHA, EPS, cfg=cfg)
        assert G.scratch_check() == (0, 0)
    q = rank.cpu().numpy().astype(np.float64)
    l1 = np.abs(q - ref).sum()
    assert st.status == 0 and l1 <= PR_L1_TOL, f"L1 {l1}"
    assert l1 <= st.error_bound * 1.0001 + 1e-12


def test_spread_ids_full_size_rmat22(atos):
    g = gg.rmat(22, 16, seed=1)
    cfg = atos.queue_config(worker_size=1024, fetch_size=1024, check_size=8, flags=atos.FLAG_SPREAD_IDS)
    with atos.Graph.from_csr(g) as G:
        rank, st = G.pagerank(ALPHA, EPS, cfg=cfg)
        colors, k, st_c = G.color(cfg=atos.queue_config(flags=atos.FLAG_SPREAD_IDS))
    q = rank.cpu().numpy().astype(np.float64)
    bound = oracle.pr_error_bound(g, q / q.sum(), ALPHA)
    assert st.status == 0 and bound <= PR_L1_TOL and st.error_bound <= PR_L1_TOL
    code, bad, kk = oracle.check_coloring(g, colors.cpu().numpy())
    assert st_c.status == 0 and code == 0 and k == kk


def test_recreated_graphs_reuse_pooled_memory(atos):
    """Graph objects created and destroyed in a loop (the end-to-end pattern) reuse the library's
    cached blocks; results stay right, and trimming returns the cache to the driver."""
    import ctypes
    g = gg.rmat(12, 16, seed=1)
    ref = pr_reference(g)
    flags = atos.FLAG_SPREAD_IDS
    for rep in range(3):
        with atos.Graph.from_csr(g) as G:
            rank, st = G.pagerank(ALPHA, EPS, cfg=atos.queue_config(flags=flags))
            assert np.abs(rank.cpu().numpy() - ref).sum() <= PR_L1_TOL, f"rep {rep}"
            colors, k, _ = G.color(cfg=atos.queue_config(flags=flags))
            assert oracle.check_coloring(g, colors.cpu().numpy())[0] == 0
            d, _ = G.bfs([0])
            assert np.array_equal(d.cpu().numpy()[0], oracle.bfs(g, 0))
    cached = ctypes.c_int64(-1)
    assert atos.abi.lib().atos_pool_trim(ctypes.byref(cached)) == 0
    assert cached.value > 0
    assert atos.abi.lib().atos_pool_trim(ctypes.byref(cached)) == 0 and cached.value == 0


@pytest.mark.parametrize("gname", list(small_graphs().keys()))
def test_color_ordered_all_configs(atos, graphs, gname):
    """ATOS_FLAG_GC_ORDERED (assigns avoid only smaller neighbours' colours): proper, within the
    first-fit range, on both layouts and every configuration; on RMAT 12 the count stays within a
    few colours of serial first fit in id order."""
    g = graphs[gname]
    _, greedy = oracle.greedy_color(g)
    with atos.Graph.from_csr(g) as G:
        for cname, cfg in configs(atos).items():
            for extra in (0, atos.FLAG_SPREAD_IDS):
                cfg.flags = atos.FLAG_GC_ORDERED | extra
                colors, k, st = G.color(cfg=cfg)
                code, bad, kk = oracle.check_coloring(g, colors.cpu().numpy())
                assert st.status == 0 and code == 0 and k == kk, f"{gname}/{cname}/{extra}: code {code} vertex {bad}"
                if gname == "rmat12" and not extra and not cname.startswith("bsp"):
                    assert k <= greedy + 4, f"{cname}: {k} colours, serial greedy {greedy}"


def test_throughput_timeline(atos):
    """atos_timeline: the per-bucket tasks and neighbour entries of a run add up to its counters,
    for the persistent and the discrete strategy; turning it off stops the recording."""
    g = gg.rmat(12, 16, seed=1)
    with atos.Graph.from_csr(g) as G:
        G.timeline(bucket_us=50.0, nbuckets=64)
        for cfg in (atos.queue_config(), atos.queue_config("discrete-cta"), atos.queue_config("persist-warp")):
            _, st = G.pagerank(ALPHA, EPS, cfg=cfg)
            tasks, edges = G.timeline_read()
            assert tasks.sum() == st.tasks and edges.sum() == st.edges and tasks.sum() > 0
            _, st = G.bfs([0, 1], cfg=cfg)
            tasks, edges = G.timeline_read()
            assert tasks.sum() == st.tasks and edges.sum() == st.edges
        G.pagerank(ALPHA, EPS, cfg=atos.queue_config("bsp"))  # BSP records nothing
        tasks, edges = G.timeline_read()
        assert tasks.sum() == 0 and edges.sum() == 0
        G.timeline()
        G.pagerank(ALPHA, EPS)


@pytest.mark.parametrize("gname", ["rmat12", "rmat11_del", "grid97x61_del", "star1000", "clique40", "two_parts",
                                   "path300", "single", "isolated3"])
def test_color_dependency_equals_serial_greedy(atos, graphs, gname):
    """ATOS_FLAG_GC_DEPENDENCY: every vertex is coloured once, after its smaller-id neighbours, so
    the colouring equals serial first fit in id order exactly -- on the input ids, and on the
    spread-id copy in that copy's id order -- for every worker shape and strategy (BSP ignores the
    flag and is checked for properness only)."""
    g = graphs[gname]
    ref, kref = oracle.greedy_color(g)
    with atos.Graph.from_csr(g) as G:
        perm, _ = G.spread_layout()
        ref_sp, kref_sp = oracle.greedy_color(g, order=np.argsort(perm))
        for cname, cfg in configs(atos).items():
            for spread in (False, True):
                cfg.flags = (cfg.flags & ~atos.FLAG_SPREAD_IDS) | atos.FLAG_GC_DEPENDENCY | (
                    atos.FLAG_SPREAD_IDS if spread else 0)
                colors, k, st = G.color(cfg=cfg)
                c = colors.cpu().numpy()
                assert st.status == 0, f"{gname}/{cname}/{spread}"
                if cname.startswith("bsp"):
                    assert oracle.check_coloring(g, c)[0] == 0
                    continue
                want, kw = (ref_sp, kref_sp) if spread else (ref, kref)
                bad = np.flatnonzero(c != want)
                assert bad.size == 0, f"{gname}/{cname}/spread={spread}: {bad.size} colours differ"
                assert k == kw
                # one release per vertex, at most one ready push, and the tail segments of the
                # rows with more than 32 larger neighbours (up to 2048 entries each)
                ids = perm if spread else np.arange(g.n)
                assert st.tasks <= 2 * g.n + _tail_segments(g, ids)
                assert G.scratch_check()[1] == 0


def _tail_segments(g, ids):
    """Tail segments the dependency-ordered colouring may create on g under the given ids."""
    deg = np.diff(g.row_ptr)
    src = np.repeat(np.arange(g.n), deg)
    larger = np.bincount(src[ids[g.col] > ids[src]], minlength=g.n) if g.n else np.zeros(0, np.int64)
    return int(np.ceil(np.maximum(0, larger - 32) / 2048).sum())


def test_color_dependency_tail_segments(atos):
    """Rows with more than 32 + 2048 larger neighbours: CTA workers hand the rest of the row,
    after the first 32, to other CTAs as tail segments of up to 2048 entries; the colouring is
    still exactly serial first fit, and the star's hub row shows up as extra tasks."""
    for g in (gg.star(20000), gg.rmat(16, 16, seed=3), _hub_ring(3, 9000)):
        ref, kref = oracle.greedy_color(g)
        with atos.Graph.from_csr(g) as G:
            for cfg in (atos.queue_config(worker_size=128, fetch_size=32, fetch_policy=atos.FETCH_GREEDY),
                        atos.queue_config(worker_size=256, fetch_size=256),
                        atos.queue_config(worker_size=1024, fetch_size=64, fetch_policy=atos.FETCH_GREEDY),
                        atos.queue_config("discrete-cta")):
                cfg.flags |= atos.FLAG_GC_DEPENDENCY
                for _ in range(2):  # the segment table is reused by the next call
                    colors, k, st = G.color(cfg=cfg)
                    assert st.status == 0 and k == kref, (g.name, cfg.worker_size)
                    assert np.array_equal(colors.cpu().numpy(), ref), (g.name, cfg.worker_size)
                    assert st.tasks <= 2 * g.n + _tail_segments(g, np.arange(g.n))
                    if g.name.startswith("star"):
                        assert st.tasks > 2 * g.n - 1, st.tasks  # the hub's tail went out as segments
            # the spread-id copy: serial first fit in that copy's id order
            perm, _ = G.spread_layout()
            ref_sp, kref_sp = oracle.greedy_color(g, order=np.argsort(perm))
            cfg = atos.queue_config(worker_size=128, fetch_size=32, fetch_policy=atos.FETCH_GREEDY,
                                    flags=atos.FLAG_GC_DEPENDENCY | atos.FLAG_SPREAD_IDS)
            colors, k, st = G.color(cfg=cfg)
            assert st.status == 0 and k == kref_sp, g.name
            assert np.array_equal(colors.cpu().numpy(), ref_sp), g.name
            assert st.tasks <= 2 * g.n + _tail_segments(g, perm)


def _hub_ring(k, leaves):
    """k hubs (ids 0..k-1) joined in a ring, each with `leaves` leaves of larger ids."""
    pairs = [(i, (i + 1) % k) for i in range(k)]
    nxt = k
    for h in range(k):
        pairs += [(h, nxt + j) for j in range(leaves)]
        nxt += leaves
    return gg.from_edges(nxt, pairs, "hub_ring")


def test_color_dependency_full_size(atos):
    """Dependency-ordered colouring on RMAT 22 (hubs have the smallest ids) and on the 2048 x 2048
    grid (its longest increasing-id path has 4094 steps): exactly serial first fit in id order."""
    for g in (gg.rmat(22, 16, seed=1), gg.grid(2048, delete_frac=0.1, seed=1)):
        ref, kref = oracle.greedy_color(g)
        with atos.Graph.from_csr(g) as G:
            colors, k, st = G.color(cfg=atos.queue_config(worker_size=512, fetch_size=512,
                                                          flags=atos.FLAG_GC_DEPENDENCY))
        assert st.status == 0 and k == kref
        assert np.array_equal(colors.cpu().numpy(), ref)


def test_color_dependency_rejected_by_batches_and_servers(atos):
    g = gg.rmat(10, 16, seed=3)
    cfg = atos.queue_config(flags=atos.FLAG_GC_DEPENDENCY)
    with atos.Graph.from_csr(g) as G:
        with pytest.raises(atos.AtosError) as e:
            atos.Batch([G], [("color", 0)], cfg)
        assert e.value.status == atos.abi.ERR_UNSUPPORTED
        with pytest.raises(atos.AtosError) as e:
            atos.Server([G], max_slots=4, budget_bytes=1 << 26, cfg=cfg)
        assert e.value.status == atos.abi.ERR_UNSUPPORTED


@pytest.mark.parametrize("gname", ["rmat12", "rmat11_del", "grid97x61_del", "star1000", "clique40", "two_parts",
                                   "path300", "single", "isolated3"])
def test_thread_workers_pagerank_and_color(atos, graphs, gname):
    """Thread workers (worker_size 1) for PageRank (Check_Size scan and threshold crossing, input
    and spread layouts) and colouring (Algorithm 6 and the dependency-ordered mode): the same
    gates as the other workers, rows longer than 32 entries handed to the warp path."""
    g = graphs[gname]
    ref = pr_reference(g)
    greedy, kg = oracle.greedy_color(g)
    with atos.Graph.from_csr(g) as G:
        for cname, cfg in thread_worker_configs(atos).items():
            for flags in (0, atos.FLAG_SPREAD_IDS, atos.FLAG_PR_CROSSING):
                cfg.flags = flags
                rank, st = G.pagerank(ALPHA, EPS, cfg=cfg)
                q = rank.cpu().numpy().astype(np.float64)
                l1 = np.abs(q - ref).sum()
                assert st.status == 0 and l1 <= PR_L1_TOL, f"{gname}/{cname}/{flags}: L1 {l1}"
                assert l1 <= st.error_bound * 1.0001 + 1e-12
                assert G.scratch_check() == (0, 0)
            for flags in (0, atos.FLAG_SPREAD_IDS, atos.FLAG_GC_ORDERED):
                cfg.flags = flags
                colors, k, st = G.color(cfg=cfg)
                code, bad, kk = oracle.check_coloring(g, colors.cpu().numpy())
                assert st.status == 0 and code == 0 and k == kk, f"{gname}/{cname}/{flags}: vertex {bad}"
            cfg.flags = atos.FLAG_GC_DEPENDENCY
            colors, k, st = G.color(cfg=cfg)
            assert st.status == 0 and k == kg and np.array_equal(colors.cpu().numpy(), greedy), f"{gname}/{cname}"


def test_thread_workers_in_batches(atos):
    """A mixed batch (BFS, PageRank, colouring over three graphs) run by thread workers: each
    result as the oracle has it."""
    gs = [gg.rmat(11, 16, seed=2), gg.grid(60, 45, delete_frac=0.1, seed=4), gg.star(300)]
    Gs = [atos.Graph.from_csr(x) for x in gs]
    specs = [("bfs", 0, 0), ("pagerank", 1), ("color", 2), ("bfs", 1, 7), ("pagerank", 0), ("color", 0)]
    for cfg in (atos.queue_config(worker_size=1, fetch_size=32), atos.queue_config("discrete-warp", worker_size=1,
                                                                                    fetch_size=16)):
        with atos.Batch(Gs, specs, cfg) as B:
            B.run()
            _, per = B.stats()
            for (kind, gi, *rest), out, st in zip(specs, B.outputs, per):
                assert st.status == 0
                x = gs[gi]
                o = out.cpu().numpy()
                if kind == "bfs":
                    assert np.array_equal(o, oracle.bfs(x, rest[0]))
                elif kind == "pagerank":
                    assert np.abs(o.astype(np.float64) - pr_reference(x)).sum() <= PR_L1_TOL
                else:
                    assert oracle.check_coloring(x, o)[0] == 0
    for G in Gs:
        G.close()
