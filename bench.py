#!/usr/bin/env python3
"""Throughput benchmark of the task-parallel scheduler on one or more GB300s.

One step = the whole hot path on one resident scale-free graph (RMAT scale 22, edge factor 16,
a, b, c = 0.57, 0.19, 0.19, seed 1): breadth-first search from 64 seeded sources in one batched
persistent launch, FP32 push-residual PageRank (alpha 0.85, eps 1e-9) and speculative greedy
colouring.  The metric is GTEPS over the step:

  * BFS: undirected edges of the source's connected component, per source (Graph500 rule);
  * PageRank: edge pushes performed (one per neighbour entry scattered to);
  * colouring: neighbour entries scanned by the assign and check tasks.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl atos|reference]
Under torchrun (N > 1) every rank runs an independent replica on its own GPU (the single-graph
path does not shard); rank 0 prints one JSON line.  ``--impl reference`` times the serial CPU
oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402

METRIC = "GTEPS (batched BFS x64 + PageRank + colouring step)"
UNIT = "GTEPS"
ALPHA, EPS = 0.85, 1e-9
NSRC = 64
L2_BYTES = 129 * 2**20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="atos", choices=["atos", "reference"])
    ap.add_argument("--scale", type=int, default=22, help="RMAT scale of the workload graph")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--worker", type=int, default=256, help="with --no-tune: worker size for every app")
    ap.add_argument("--fetch", type=int, default=256, help="with --no-tune: fetch size for every app")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner; use --worker / --fetch")
    ap.add_argument("--check-size", type=int, default=32, help="with --no-tune: PageRank's Check_Size")
    ap.add_argument("--flags", type=int, default=0, help="with --no-tune: atos_config.flags of PageRank and colouring")
    ap.add_argument("--policy", type=int, default=2, help="with --no-tune: PageRank's fetch policy (0 fixed, 1 greedy, 2 spread)")
    ap.add_argument("--no-compare", action="store_true", help="skip the BSP / unbatched comparisons")
    ap.add_argument("--cfg", action="append", default=[], metavar="APP=W,F,P,C,WIN,FLAGS[,STRATEGY]",
                    help="fix one application's configuration instead of autotuning it (app: bfs, pagerank, "
                         "color; worker, fetch, fetch policy, Check_Size, window, flags, strategy 0/1/2)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads measured beside the main step (2048^2 grid, batched mix, "
                         "serving window)")
    ap.add_argument("--study", default=None, choices=["color-ids"],
                    help="color-ids: colouring on the input ids, the spread ids and a random relabelling, for "
                         "several worker shapes and BSP (Section 6.4's permutation experiment); prints one JSON "
                         "line instead of the bench line")
    ap.add_argument("--workload", default="rmat22", choices=["rmat22", "batched"],
                    help="rmat22: the single-graph step (default); batched: 256 graphs x (4 BFS + 1 PageRank) "
                         "in one batched launch")
    return ap.parse_args()


def parse_cfgs(atos, specs):
    """{app: Config} from --cfg APP=worker,fetch,policy,check_size,window,flags[,strategy]."""
    out = {}
    for spec in specs:
        app, vals = spec.split("=", 1)
        v = [int(x) for x in vals.split(",")]
        cfg = atos.queue_config(worker_size=v[0], fetch_size=v[1], fetch_policy=v[2], check_size=v[3], window=v[4],
                                flags=v[5])
        if len(v) > 6:
            cfg.strategy = v[6]
        out[app] = cfg
    return out


def workload(scale: int):
    g = gg.rmat(scale, 16, 0.57, 0.19, 0.19, seed=1)
    srcs = gg.sources(g, NSRC, seed=1)
    return g, srcs


def workload_config(g, args, extra=None):
    cfg = {"workload": f"rmat{args.scale}_bfs{NSRC}_pagerank_color", "graph": f"RMAT scale {args.scale}, edge "
           f"factor 16, a=0.57 b=0.19 c=0.19, seed 1, symmetrised, deduplicated", "n": g.n, "nnz": g.nnz,
           "bfs_sources": NSRC, "alpha": ALPHA, "eps": EPS,
           "l2": (f"inputs larger than L2: col is {g.nnz * 4 / 2**20:.0f} MiB vs 129 MiB L2 (no flush needed)"
                  if 4 * g.nnz > L2_BYTES else "inputs smaller than L2 (not flushed between steps)")}
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------------------------ clocks

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[4:8]):
                if flag.lower() in ("active", "1", "0x1"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- replicas (N > 1)

def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest replica's time: every rank contributes its own timed-region length and all get
    the maximum (the job is done when the last replica is)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(work_per_replica: float, total_ms: float, steps: int, world: int):
    """(ms per step, whole-job GTEPS): `world` independent replicas each did `work_per_replica`
    edges per step; the job took the slowest replica's time (weak scaling)."""
    ms_step = total_ms / steps
    return ms_step, world * work_per_replica / (ms_step * 1e-3) / 1e9


TRAFFIC_SOURCES = ("engine.cuh", "pagerank.cuh", "pagerank.cu", "relabel.cu")


def kernel_sources_digest(src_dir=None):
    """sha256 of the PageRank kernel's sources with comments and whitespace removed, so that only a
    change of the code itself voids the recorded traffic."""
    import hashlib
    import re
    src_dir = src_dir or os.path.join(ROOT, "paper_2112_00132_gb300", "csrc")
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        text = open(os.path.join(src_dir, f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)  # block comments
        text = re.sub(r"//[^\n]*", " ", text)                # line comments
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def recorded_traffic(cfg_pr, path=None, src_dir=None):
    """DRAM bytes per launch of the PageRank kernel from the committed ncu record, or None when
    the kernel's code changed since it was taken or the configuration differs."""
    path = path or os.path.join(ROOT, "profiles", "pagerank_traffic_rmat22.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    digest = [ln.split(": ", 1)[1].strip() for ln in lines if ln.startswith("kernel_code_sha256: ")]
    if not digest or digest[0] != kernel_sources_digest(src_dir):
        return None
    key = (cfg_pr.worker_size, cfg_pr.fetch_size, cfg_pr.fetch_policy, cfg_pr.check_size, cfg_pr.flags)
    for ln in lines:
        if ln.startswith("entry: "):
            fields = ln.split()[1:]
            if tuple(int(x) for x in fields[:5]) == key:
                return float(fields[5])
    return None


# ------------------------------------------------------------------------------- atos arm

def component_edges(depths, deg_t):
    """Graph500 edge count per BFS: undirected edges with both ends reached (sum of reached
    degrees / 2), from the depths on the device."""
    import torch
    reached = depths != 2**31 - 1
    return (reached.to(torch.int64) * deg_t.unsqueeze(0)).sum(dim=1) // 2


def run_atos(args, rank: int, world: int):
    import torch

    import paper_2112_00132_gb300 as atos

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    atos.build() if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    atos.lib()
    g, srcs = workload(args.scale)
    stream = torch.cuda.current_stream()
    G = atos.Graph.from_csr(g, skip_validation=False)
    depths = torch.empty((NSRC, g.n), dtype=torch.int32, device="cuda")
    rank_t = torch.empty(g.n, dtype=torch.float32, device="cuda")
    colors = torch.empty(g.n, dtype=torch.int32, device="cuda")
    deg_t = torch.from_numpy(np.diff(g.row_ptr).astype(np.int64)).cuda()

    # configuration per application: the autotuner's choice (untimed sweep), unless fixed
    if args.no_tune:
        cfg_bfs = atos.queue_config(worker_size=args.worker, fetch_size=args.fetch)
        cfg_gc = atos.queue_config(worker_size=args.worker, fetch_size=args.fetch, flags=args.flags)
        cfg_pr = atos.queue_config(worker_size=args.worker, fetch_size=args.fetch, check_size=args.check_size,
                                   flags=args.flags, fetch_policy=args.policy)
        tune_ms = {}
    else:
        fixed = parse_cfgs(atos, args.cfg)
        tune_ms = {}
        if "bfs" in fixed:
            cfg_bfs = fixed["bfs"]
        else:
            cfg_bfs, t_b = G.autotune("bfs", srcs, repeats=1, stream=stream)
            tune_ms["bfs"] = round(t_b, 3)
        if "pagerank" in fixed:
            cfg_pr = fixed["pagerank"]
        else:
            cfg_pr, t_p = G.autotune("pagerank", repeats=1, stream=stream)
            tune_ms["pagerank"] = round(t_p, 3)
        if "color" in fixed:
            cfg_gc = fixed["color"]
        else:
            cfg_gc, t_c = G.autotune("color", repeats=1, stream=stream)
            tune_ms["color"] = round(t_c, 3)

    # warm-up steps with statistics (synchronising), to count the work of a step
    bfs_edges = pr_edges = gc_edges = 0
    pr_tasks = 0
    bfs_stats = pr_stats = gc_stats = None
    for w in range(max(args.warmup, 3)):
        _, bfs_stats = G.bfs(srcs, depths, cfg=cfg_bfs, stream=stream)
        _, pr_stats = G.pagerank(ALPHA, EPS, rank_t, cfg=cfg_pr, stream=stream)
        _, ncol, gc_stats = G.color(colors, cfg=cfg_gc, stream=stream)
        pr_edges += pr_stats.edges
        pr_tasks += pr_stats.tasks
        gc_edges += gc_stats.edges
    nw = max(args.warmup, 3)
    pr_edges /= nw
    pr_tasks /= nw
    gc_edges /= nw
    comp = component_edges(depths, deg_t)
    bfs_edges = int(comp.sum().item())
    reached_v = int((depths != 2**31 - 1).sum().item())
    comp_nnz = 2 * bfs_edges

    # timed steps: no statistics, no host synchronisation inside a step
    l0 = atos.kernel_launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clocks:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        step_ev = []
        for s in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e3 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.bfs(srcs, depths, cfg=cfg_bfs, stream=stream, stats=False)
            e1.record(stream)
            G.pagerank(ALPHA, EPS, rank_t, cfg=cfg_pr, stream=stream, stats=False)
            e2.record(stream)
            G.color(colors, cfg=cfg_gc, stream=stream, stats=False)
            e3.record(stream)
            step_ev.append((e0, e1, e2, e3))
        t_end.record(stream)
        torch.cuda.synchronize()
    launches = atos.kernel_launches() - l0
    total_ms = t_start.elapsed_time(t_end)
    bfs_ms = [a.elapsed_time(b) for a, b, _, _ in step_ev]
    pr_ms = [b.elapsed_time(c) for _, b, c, _ in step_ev]
    gc_ms = [c.elapsed_time(d) for _, _, c, d in step_ev]
    total_ms = max_over_ranks(total_ms, world, "cuda")
    if world > 1:
        torch.distributed.barrier()
    work = bfs_edges + pr_edges + gc_edges
    ms_step, value = replica_throughput(work, total_ms, args.steps, world)

    # roofline of the dominant kernel (the call whose kernels take the most time)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    mean = lambda xs: sum(xs) / len(xs)  # noqa: E731
    pct = lambda xs, q: float(np.percentile(np.asarray(xs), q))  # noqa: E731
    parts = {
        # bytes per launch: PageRank 20 B per push + 8 B per edge push (a col read and a residue
        # update); BFS, per source, 8 B per component entry (col read + neighbour depth read) +
        # 12 B per vertex (row_ptr, depth init and final write); colouring 16 B per entry + 24 B
        # per vertex (assign + check passes)
        "pagerank_persistent": (mean(pr_ms), 20.0 * pr_tasks + 8.0 * pr_edges),
        "bfs_persistent_batched": (mean(bfs_ms), NSRC * 12.0 * g.n + 8.0 * comp_nnz),
        "color_persistent": (mean(gc_ms), 16.0 * g.nnz + 24.0 * g.n),
    }
    dom = max(parts, key=lambda k: parts[k][0])
    dom_ms, dom_bytes = parts[dom]
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    traffic = recorded_traffic(cfg_pr) if (dom == "pagerank_persistent" and args.scale == 22
                                           and cfg_pr.strategy == 0) else None
    roofline = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "peak_source": peak_src, "traffic": traffic,
                "traffic_source": "profiles/pagerank_traffic_rmat22.txt (ncu, one launch)" if traffic else None,
                "algorithmic_bytes": dom_bytes, "launch_ms": round(dom_ms, 3)}
    # the edge-loop ceilings on this graph (library probe, no scheduler): the rate the bodies'
    # inner loops could reach; the kernels are bound by L2 atomics and gather latency, not HBM
    # throughput over one PageRank run (the paper's throughput-vs-time view), outside the timed steps
    nb = 24
    bucket_us = max(1.0, mean(pr_ms) * 1e3 / (nb - 4))
    G.timeline(bucket_us=bucket_us, nbuckets=nb)
    G.pagerank(ALPHA, EPS, rank_t, cfg=cfg_pr, stream=stream, stats=False)
    tl_tasks, tl_edges = G.timeline_read()
    G.timeline()
    pagerank_timeline = {"bucket_ms": round(bucket_us / 1e3, 3),
                         "g_edge_pushes_per_s": [round(float(e) / (bucket_us * 1e-6) / 1e9, 1) for e in tl_edges],
                         "tasks": [int(t) for t in tl_tasks]}
    # each on the layout the application ran on (spread ids when its configuration says so)
    def ceiling(kind, spread):
        return g.nnz / G.edge_ceiling(kind, repeats=3, stream=stream, spread_ids=spread) / 1e6
    pr_spread, gc_spread = bool(cfg_pr.flags & atos.FLAG_SPREAD_IDS), bool(cfg_gc.flags & atos.FLAG_SPREAD_IDS)
    scatter_g = ceiling("scatter", pr_spread)
    gather_bfs_g = ceiling("gather", False)
    gather_gc_g = ceiling("gather", gc_spread)
    bfs_reads = float(bfs_stats.edges)
    rate = lambda work, ms: work / (mean(ms) * 1e-3) / 1e9  # noqa: E731
    edge_ceiling = {
        "unit": "G edge operations/s",
        "pagerank": {"achieved": round(rate(pr_edges, pr_ms), 1), "ceiling": round(scatter_g, 1),
                     "frac": round(rate(pr_edges, pr_ms) / scatter_g, 3), "layout": "spread" if pr_spread else "input"},
        "bfs": {"achieved": round(rate(bfs_reads, bfs_ms), 1), "ceiling": round(gather_bfs_g, 1),
                "frac": round(rate(bfs_reads, bfs_ms) / gather_bfs_g, 3), "layout": "input"},
        "color": {"achieved": round(rate(gc_edges, gc_ms), 1), "ceiling": round(gather_gc_g, 1),
                  "frac": round(rate(gc_edges, gc_ms) / gather_gc_g, 3), "layout": "spread" if gc_spread else "input"},
        "probe": "atos_edge_ceiling: one pass over every CSR entry in order, col[e] then red.add.f32 (PageRank: "
                 "scatter) or a load (BFS, colouring: gather) of state[col[e]], on the application's layout; "
                 "BFS and colouring work counted as neighbour entries read",
    }

    def brief(c):
        names = {0: "persistent", 1: "discrete", 2: "bsp"}
        return {"worker": c.worker_size, "fetch": c.fetch_size, "strategy": names.get(c.strategy, c.strategy),
                "fetch_policy": c.fetch_policy, "window": c.window, "check_size": c.check_size, "flags": c.flags}

    # comparators (untimed by the step, timed here with the same events): the level-synchronous
    # BSP forms (host-driven levels, levels in a device-side graph loop; BFS one source at a time
    # and all 64 at once) and the unbatched single-query form of the same work
    comparisons = {}
    if not args.no_compare:
        comparisons = compare_rmat(atos, G, g, srcs, depths, rank_t, colors, stream,
                                   dict(cfg_bfs=cfg_bfs, cfg_pr=cfg_pr, cfg_gc=cfg_gc, bfs_ms=bfs_ms, pr_ms=pr_ms,
                                        gc_ms=gc_ms, ms_step=ms_step, bfs_edges=bfs_edges, pr_edges=pr_edges,
                                        gc_edges=gc_edges, bfs_stats=bfs_stats, ncol=int(ncol)))

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32 (BFS, colouring) + f32 (PageRank)", "data": "synthetic",
        "config": workload_config(g, args, {"bfs_cfg": brief(cfg_bfs), "pagerank_cfg": brief(cfg_pr),
                                            "color_cfg": brief(cfg_gc), "autotuned": not args.no_tune,
                                            "autotune_best_ms": tune_ms, "parallelism": f"replicas x{world}"}),
        "comparisons": comparisons,
        "roofline": roofline,
        "edge_ceiling": edge_ceiling,
        "pagerank_timeline": pagerank_timeline,
        "gpu_launches": launches,
        "breakdown": {
            "bfs_ms": round(mean(bfs_ms), 3), "pagerank_ms": round(mean(pr_ms), 3), "color_ms": round(mean(gc_ms), 3),
            "p50_ms": {k: round(pct(v, 50), 3) for k, v in (("bfs", bfs_ms), ("pagerank", pr_ms), ("color", gc_ms))},
            "p99_ms": {k: round(pct(v, 99), 3) for k, v in (("bfs", bfs_ms), ("pagerank", pr_ms), ("color", gc_ms))},
            "bfs_gteps": round(bfs_edges / (mean(bfs_ms) * 1e-3) / 1e9, 3),
            "pagerank_gteps": round(pr_edges / (mean(pr_ms) * 1e-3) / 1e9, 3),
            "color_gteps": round(gc_edges / (mean(gc_ms) * 1e-3) / 1e9, 3),
            "bfs_graph500_edges": bfs_edges, "bfs_reached_vertices": reached_v, "bfs_tasks": bfs_stats.tasks,
            "pagerank_edge_pushes": pr_edges, "pagerank_tasks": pr_tasks,
            "pagerank_error_bound": pr_stats.error_bound, "color_edges": gc_edges, "colors": int(ncol),
            # Table 4's colouring measure: tasks relative to the vertex count (an assign and a
            # check task per vertex at least, so 2.0 means no recolouring)
            "color_tasks_per_vertex": round(gc_stats.tasks / g.n, 4),
        },
        "clocks": clocks.summary(),
    }
    # the end-to-end leg builds its own graph objects: release this one (and its autotuning and
    # comparison state, CUDA graphs of the device-loop BSP forms included) first
    G.close()
    del depths
    torch.cuda.synchronize()
    if not args.no_e2e:
        result["e2e"] = run_e2e(args, g, srcs, (cfg_bfs, cfg_pr, cfg_gc), bfs_edges + pr_edges + gc_edges, world)
    if not args.no_configs and world == 1:
        # the other workloads, each measured on its own after the main step (not part of `value`)
        result["configs"] = {"grid2048": grid_leg(atos, stream, dev, hbm_peak),
                             "batched": batched_leg(atos, stream, dev, hbm_peak),
                             "serving": serving_leg(atos, dev)}
    return result


def timed_ms(fn, stream, reps=2):
    """Device time of one call of fn on `stream` (CUDA events, after one untimed call), median of
    `reps` calls."""
    import torch
    fn()
    out = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
    return statistics.median(out)


def bsp_configs(atos):
    """The level-synchronous forms: levels driven by the host, or looped on the device in a CUDA
    graph's conditional node."""
    q = atos.queue_config
    return {"host": q("bsp"), "device_loop": q("bsp", flags=atos.FLAG_BSP_DEVICE_LOOP)}


def compare_rmat(atos, G, g, srcs, depths, rank_t, colors, stream, m):
    """The persistent step against the project's level-synchronous (BSP) forms and the unbatched
    single-query form, application by application, with Table 4's workload ratio and the paper's
    normalised throughput (useful work, counted as the BSP form's work, per second)."""
    import torch
    q = atos.queue_config
    mean = lambda xs: sum(xs) / len(xs)  # noqa: E731
    out = {}
    # BFS x 64; the unbatched single-query form with the configuration the autotuner picks for one
    # source (the tuned multi-source one is shaped for 64 searches at once)
    one = torch.empty((1, g.n), dtype=torch.int32, device="cuda")
    cfg_one, _ = G.autotune("bfs", [int(srcs[0])], repeats=1, stream=stream)

    def unbatched():
        for s0 in srcs:
            G.bfs([int(s0)], one, cfg=cfg_one, stream=stream, stats=False)
    bfs = {"persistent_batched_ms": round(mean(m["bfs_ms"]), 3),
           "persistent_unbatched_ms": round(timed_ms(unbatched, stream, reps=1), 3),
           "unbatched_cfg": cfg_brief(cfg_one)}
    for name, cfg in bsp_configs(atos).items():
        # sources in groups that keep their depth arrays L2-resident (the default), and all at once
        bfs[f"bsp_grouped_{name}_ms"] = round(timed_ms(
            lambda: G.bfs(srcs, depths, cfg=cfg, stream=stream, stats=False), stream), 3)
        every = q("bsp", flags=cfg.flags, window=len(srcs))
        bfs[f"bsp_all_sources_{name}_ms"] = round(timed_ms(
            lambda: G.bfs(srcs, depths, cfg=every, stream=stream, stats=False), stream, reps=1), 3)
    per_source = q("bsp", flags=atos.FLAG_BSP_PER_SOURCE)
    bfs["bsp_per_source_host_ms"] = round(timed_ms(
        lambda: G.bfs(srcs, depths, cfg=per_source, stream=stream, stats=False), stream, reps=1), 3)
    bfs["best_bsp_ms"] = min(v for k, v in bfs.items() if k.startswith("bsp_"))
    bfs["unbatched_vs_bsp_per_source"] = round(bfs["bsp_per_source_host_ms"] / bfs["persistent_unbatched_ms"], 3)
    _, bsp_bfs = G.bfs(srcs, depths, cfg=q("bsp"), stream=stream)
    bfs["bsp_levels"] = int(bsp_bfs.iterations)
    out["bfs64"] = bfs
    # PageRank and colouring: each BSP form at its better layout (input or spread ids)
    def best_bsp(run):
        best = None
        for name, base in bsp_configs(atos).items():
            for layout, flags in (("input", 0), ("spread", atos.FLAG_SPREAD_IDS)):
                cfg = q("bsp", flags=base.flags | flags)
                t = timed_ms(lambda: run(cfg), stream)
                if best is None or t < best[0]:
                    best = (t, name, layout, cfg)
                out.setdefault("_bsp_times", {})[f"{run.__name__}_{name}_{layout}"] = round(t, 3)
        return best

    def pagerank(cfg):
        G.pagerank(ALPHA, EPS, rank_t, cfg=cfg, stream=stream, stats=False)

    def color(cfg):
        G.color(colors, cfg=cfg, stream=stream, stats=False)
    t_pr, form_pr, lay_pr, cfg_bsp_pr = best_bsp(pagerank)
    t_gc, form_gc, lay_gc, cfg_bsp_gc = best_bsp(color)
    bsp_times = out.pop("_bsp_times")
    _, bsp_pr_st = G.pagerank(ALPHA, EPS, rank_t, cfg=cfg_bsp_pr, stream=stream)
    _, k_bsp, bsp_gc_st = G.color(colors, cfg=cfg_bsp_gc, stream=stream)
    out["pagerank"] = {"persistent_ms": round(mean(m["pr_ms"]), 3), "best_bsp_ms": round(t_pr, 3),
                       "best_bsp_form": f"{form_pr}, {lay_pr} ids", "bsp_levels": int(bsp_pr_st.iterations),
                       "bsp_error_bound": bsp_pr_st.error_bound,
                       **{k.split("_", 1)[1] + "_ms": v for k, v in bsp_times.items() if k.startswith("pagerank_")}}
    # colouring: the tuned run against the BSP form, the fastest speculative run of Algorithm 6
    # and the ordered variant, each with its colour count
    spec_cfg = q(worker_size=512, fetch_size=512, flags=atos.FLAG_SPREAD_IDS)
    t_spec = timed_ms(lambda: color(spec_cfg), stream)
    _, k_spec, st_spec = G.color(colors, cfg=spec_cfg, stream=stream)
    ordered = q(worker_size=512, fetch_size=512, flags=atos.FLAG_GC_ORDERED)
    _, k_ord, st_ord = G.color(colors, cfg=ordered, stream=stream)
    out["color"] = {"persistent_ms": round(mean(m["gc_ms"]), 3), "persistent_colors": m["ncol"],
                    "persistent_dependency_ordered": bool(m["cfg_gc"].flags & atos.FLAG_GC_DEPENDENCY),
                    "best_bsp_ms": round(t_gc, 3), "best_bsp_form": f"{form_gc}, {lay_gc} ids",
                    "bsp_colors": int(k_bsp), "bsp_levels": int(bsp_gc_st.iterations),
                    **{k.split("_", 1)[1] + "_ms": v for k, v in bsp_times.items() if k.startswith("color_")},
                    "speculative_cta512_spread": {"ms": round(t_spec, 3), "colors": int(k_spec),
                                                  "tasks_per_vertex": round(st_spec.tasks / g.n, 3)},
                    "ordered_cta512": {"ms": round(st_ord.ms, 3), "colors": int(k_ord),
                                       "tasks_per_vertex": round(st_ord.tasks / g.n, 3)}}
    best_step = bfs["best_bsp_ms"] + t_pr + t_gc
    out["step"] = {"persistent_ms": round(m["ms_step"], 3), "best_bsp_ms": round(best_step, 3),
                   "speedup_vs_best_bsp": round(best_step / m["ms_step"], 3),
                   "note": "best BSP form per application (host- or device-driven levels, all sources at once or "
                           "one at a time, input or spread ids) against the persistent step"}
    out["workload_ratio"] = {
        "bfs": round(m["bfs_stats"].edges / max(1, bsp_bfs.edges), 3),
        "pagerank": round(m["pr_edges"] / max(1, bsp_pr_st.edges), 3),
        "color": round(m["gc_edges"] / max(1, bsp_gc_st.edges), 3),
        "note": "neighbour entries read by the persistent path / by the BSP path (Table 4's ratio)"}
    useful = {"bfs": m["bfs_edges"], "pagerank": float(bsp_pr_st.edges), "color": float(bsp_gc_st.edges)}
    times = {"bfs": mean(m["bfs_ms"]), "pagerank": mean(m["pr_ms"]), "color": mean(m["gc_ms"])}
    out["normalized_gteps"] = {
        **{k: round(useful[k] / (times[k] * 1e-3) / 1e9, 3) for k in useful},
        "step": round(sum(useful.values()) / (m["ms_step"] * 1e-3) / 1e9, 3),
        "note": "Section 6's normalised throughput: useful work per second, the useful work of PageRank and "
                "colouring counted as the BSP form's edge work (BFS: Graph500 edges, as the headline)"}
    return out


def _pcts(xs):
    return {"p50_ms": round(float(np.percentile(xs, 50)), 3), "p99_ms": round(float(np.percentile(xs, 99)), 3),
            "mean_ms": round(float(np.mean(xs)), 3)}


def _device_times(fn, stream, runs):
    """Per-call device times (CUDA events on `stream`) of `runs` calls of fn after one warm-up."""
    import torch
    fn()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(runs + 1)]
    evs[0].record(stream)
    for k in range(runs):
        fn()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    return [evs[k].elapsed_time(evs[k + 1]) for k in range(runs)]


def grid_leg(atos, stream, dev, hbm_peak, runs=10):
    """The high-diameter mesh: a 2048 x 2048 4-neighbour grid with 10% of its edges deleted
    (seed 1), BFS from the corner vertex and FP32 PageRank, each autotuned, against the best BSP
    form (levels driven by the host or looped on the device; PageRank at its better layout)."""
    import torch
    g = gg.grid(2048, delete_frac=0.1, seed=1)
    G = atos.Graph.from_csr(g)
    q = atos.queue_config
    depth = torch.empty((1, g.n), dtype=torch.int32, device="cuda")
    rank = torch.empty(g.n, dtype=torch.float32, device="cuda")
    cfg_b, _ = G.autotune("bfs", [0], repeats=1, stream=stream)
    cfg_p, _ = G.autotune("pagerank", repeats=1, stream=stream)
    _, st_b = G.bfs([0], depth, cfg=cfg_b, stream=stream)
    _, st_p = G.pagerank(ALPHA, EPS, rank, cfg=cfg_p, stream=stream)
    deg = torch.from_numpy(np.diff(g.row_ptr).astype(np.int64)).cuda()
    comp = int(component_edges(depth, deg).sum().item())
    with ClockSampler(dev) as clocks:
        bfs_ms = _device_times(lambda: G.bfs([0], depth, cfg=cfg_b, stream=stream, stats=False), stream, runs)
        pr_ms = _device_times(lambda: G.pagerank(ALPHA, EPS, rank, cfg=cfg_p, stream=stream, stats=False), stream,
                              runs)
    bfs = {"graph500_edges": comp, "gteps": round(comp / (np.mean(bfs_ms) * 1e-3) / 1e9, 3), **_pcts(bfs_ms),
           "tasks": st_b.tasks, "cfg": cfg_brief(cfg_b)}
    for name, cfg in bsp_configs(atos).items():
        _, st = G.bfs([0], depth, cfg=cfg, stream=stream)
        bfs[f"bsp_{name}_ms"] = round(min(st.ms, timed_ms(
            lambda: G.bfs([0], depth, cfg=cfg, stream=stream, stats=False), stream, reps=1)), 3)
        bfs["bsp_levels"] = int(st.iterations)
    bfs["speedup_vs_best_bsp"] = round(min(bfs["bsp_host_ms"], bfs["bsp_device_loop_ms"]) / np.mean(bfs_ms), 3)
    pr = {"edge_pushes": st_p.edges, "tasks": st_p.tasks,
          "g_edge_pushes_per_s": round(st_p.edges / (np.mean(pr_ms) * 1e-3) / 1e9, 3), **_pcts(pr_ms),
          "error_bound": st_p.error_bound, "cfg": cfg_brief(cfg_p)}
    best = None
    for name, base in bsp_configs(atos).items():
        for layout, flags in (("input", 0), ("spread", atos.FLAG_SPREAD_IDS)):
            cfg = q("bsp", flags=base.flags | flags)
            t = timed_ms(lambda: G.pagerank(ALPHA, EPS, rank, cfg=cfg, stream=stream, stats=False), stream, reps=1)
            pr[f"bsp_{name}_{layout}_ms"] = round(t, 3)
            best = t if best is None else min(best, t)
    pr["speedup_vs_best_bsp"] = round(best / np.mean(pr_ms), 3)
    # PageRank's algorithmic bytes (20 B per task + 8 B per edge push) against the measured HBM peak
    pr["roofline_frac"] = round((20.0 * st_p.tasks + 8.0 * st_p.edges) / (np.mean(pr_ms) * 1e-3) / 1e9 / hbm_peak, 4)
    G.close()
    return {"workload": "grid2048_del0.1_bfs0_pagerank", "graph": "2048 x 2048 4-neighbour grid, 10% of edges "
            "deleted (seed 1), row-major ids", "n": g.n, "nnz": g.nnz, "bfs": bfs, "pagerank": pr,
            "runs": runs, "clocks": clocks.summary()}


def batched_leg(atos, stream, dev, hbm_peak, runs=5):
    """The batched mix (256 graphs, 1024 BFS + 256 PageRank instances) in one persistent launch
    replayed as a CUDA graph, with the configuration the batch autotuner chose on this mix
    (512-thread CTAs, fetch 512, window 512, Check_Size 8, spread ids; `bench.py --workload
    batched` reruns the sweep), against the same work as per-graph calls."""
    import torch
    graphs, specs = batched_workload()
    Gs = [atos.Graph.from_csr(x) for x in graphs]
    cfg = atos.queue_config(worker_size=512, fetch_size=512, window=512, check_size=8, flags=atos.FLAG_SPREAD_IDS)
    B = atos.Batch(Gs, specs, cfg)
    B.run(stream=stream, graph=True)
    B.run(stream=stream, graph=True)
    _, per = B.stats(stream=stream)
    bfs_edges = pr_edges = pr_tasks = 0
    bfs_bytes = 0.0
    ok = True
    for (kind, gi, *rest), out, st in zip(specs, B.outputs, per):
        ok &= st.status == 0
        x = graphs[gi]
        if kind == "bfs":
            deg = torch.from_numpy(np.diff(x.row_ptr).astype(np.int64)).cuda()
            comp = int(((out != 2**31 - 1).to(torch.int64) * deg).sum().item())
            bfs_edges += comp // 2
            bfs_bytes += 12.0 * x.n + 8.0 * comp
        else:
            pr_edges += st.edges
            pr_tasks += st.tasks
    with ClockSampler(dev) as clocks:
        ms = _device_times(lambda: B.run(stream=stream, graph=True), stream, runs)
    outs = [(torch.empty((BATCH_BFS, x.n), dtype=torch.int32, device="cuda"),
             torch.empty(x.n, dtype=torch.float32, device="cuda")) for x in graphs]
    srcs = [[sp[2] for sp in specs if sp[0] == "bfs" and sp[1] == gi] for gi in range(len(graphs))]

    def per_graph():
        for gi, G in enumerate(Gs):
            G.bfs(srcs[gi], outs[gi][0], cfg=cfg, stream=stream, stats=False)
            G.pagerank(ALPHA, EPS, outs[gi][1], cfg=cfg, stream=stream, stats=False)
    t_calls = timed_ms(per_graph, stream, reps=1)
    work = bfs_edges + pr_edges
    algo = bfs_bytes + 20.0 * pr_tasks + 8.0 * pr_edges
    res = {"workload": "batched_mix_256g_bfs4_pr1", "graphs": "128 RMAT (scale U{10..18}) + 128 grids (side "
           "U{64..1024}), 10% edge deletion, seed 1", "instances": len(specs), "all_ok": bool(ok),
           "gteps": round(work / (np.mean(ms) * 1e-3) / 1e9, 3), **_pcts(ms),
           "per_graph_calls_ms": round(t_calls, 3), "speedup_vs_per_graph_calls": round(t_calls / np.mean(ms), 3),
           "roofline": {"bound": "hbm", "achieved": round(algo / (np.mean(ms) * 1e-3) / 1e9, 1), "peak": hbm_peak,
                        "unit": "GB/s", "frac": round(algo / (np.mean(ms) * 1e-3) / 1e9 / hbm_peak, 4)},
           "bfs_graph500_edges": bfs_edges, "pagerank_edge_pushes": pr_edges, "cfg": cfg_brief(cfg),
           "window": B.window, "cuda_graph": True, "runs": runs, "clocks": clocks.summary()}
    B.close()
    for G in Gs:
        G.close()
    return res


def serving_leg(atos, dev, duration=4.0):
    """A bounded serving window: 64 resident graphs of the batched mix plus RMAT 23, Poisson
    arrivals (BFS 60%, PageRank 30%, colouring 10%), admitted by footprint; offered at the 2000
    req/s of the serving configuration and at 100 req/s.  Latency = completion - arrival."""
    from paper_2112_00132_gb300 import serve as srv
    csrs = srv.config_graphs()
    graphs = [atos.Graph.from_csr(x) for x in csrs]
    keys = ("offered_rps", "achieved_rps", "sustainable", "requests", "completed", "unfinished", "p50_ms", "p99_ms",
            "p50_ms_by_kind", "p99_ms_by_kind", "gteps", "epochs", "wall_s")
    out = {"workload": "serving: 64 graphs drawn from the batched mix + RMAT 23, Poisson arrivals, mix BFS 60% / "
           "PageRank 30% / colouring 10%", "window_s": duration, "warmup_s": 1.0}
    with ClockSampler(dev) as clocks:
        for rate in (2000.0, 100.0):
            r = srv.serve(csrs, rate=rate, duration=duration, warmup=1.0, drain_s=6.0, graphs=graphs)
            out[f"offered_{int(rate)}"] = {k: r[k] for k in keys}
    out["clocks"] = clocks.summary()
    for G in graphs:
        G.close()
    return out


def cfg_brief(c):
    names = {0: "persistent", 1: "discrete", 2: "bsp"}
    return {"worker": c.worker_size, "fetch": c.fetch_size, "strategy": names.get(c.strategy, c.strategy),
            "fetch_policy": c.fetch_policy, "window": c.window, "check_size": c.check_size, "flags": c.flags}


def run_color_ids_study(args):
    """Colouring time, recolouring work and colour count on three vertex-id layouts of the same
    graph: the generator's ids (neighbours have close ids), the library's spread ids
    (ATOS_FLAG_SPREAD_IDS) and a seeded uniform random relabelling.  Section 6.4 attributes the
    colouring overwork to neighbours sitting next to each other in the initial queue and removes it
    with a random permutation; this measures the same on the RMAT 22 bench graph and the 2048 x 2048
    grid.  Work is colour assignments per vertex (1.0: nobody recoloured)."""
    import torch

    import paper_2112_00132_gb300 as atos

    atos.build()
    atos.lib()
    q = atos.queue_config
    impls = {"discrete-warp": ("discrete-warp", {}), "persist-warp": ("persist-warp", {}),
             "persist-cta512": (None, {"worker_size": 512, "fetch_size": 512}), "bsp": ("bsp", {})}
    out = {"study": "color_id_layout", "unit": "ms", "runs": 3, "graphs": {}}
    for gname, g in (("rmat22", workload(args.scale)[0]), ("grid2048_del0.1", gg.grid(2048, delete_frac=0.1, seed=1))):
        rel, _ = gg.relabel(g, seed=1)
        res = {"n": g.n, "nnz": g.nnz}
        for layout, graph, flags in (("input", g, 0), ("spread", g, atos.FLAG_SPREAD_IDS), ("random", rel, 0)):
            G = atos.Graph.from_csr(graph)
            colors = torch.empty(g.n, dtype=torch.int32, device="cuda")
            row = {}
            for iname, (preset, kw) in impls.items():
                cfg = q(preset, flags=flags, **kw)
                G.color(colors, cfg=cfg)  # warm-up
                runs = [G.color(colors, cfg=cfg) for _ in range(3)]
                ms = sorted(r[2].ms for r in runs)
                k, st = runs[-1][1], runs[-1][2]
                assign = st.tasks / g.n if iname == "bsp" else st.tasks / (2 * g.n)
                row[iname] = {"ms": round(ms[1], 3), "assign_per_vertex": round(assign, 4), "colors": int(k)}
            res[layout] = row
            G.close()
            torch.cuda.synchronize()
        out["graphs"][gname] = res
    return out


def run_e2e(args, g, srcs, cfgs, work, world):
    """The same step through the public API from pinned host buffers: upload the CSR, run the
    three calls, read the results back, destroy the graph."""
    import torch

    import paper_2112_00132_gb300 as atos
    stream = torch.cuda.current_stream()
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    depths_h = torch.empty((NSRC, g.n), dtype=torch.int32).pin_memory()
    rank_h = torch.empty(g.n, dtype=torch.float32).pin_memory()
    colors_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
    depths = torch.empty((NSRC, g.n), dtype=torch.int32, device="cuda")
    rank_t = torch.empty(g.n, dtype=torch.float32, device="cuda")
    colors = torch.empty(g.n, dtype=torch.int32, device="cuda")

    cfg_bfs, cfg_pr, cfg_gc = cfgs
    copy_stream = torch.cuda.Stream()

    def step():
        G = atos.Graph(rp_h.numpy(), col_h.numpy(), skip_validation=True, stream=stream)
        G.bfs(srcs, depths, cfg=cfg_bfs, stream=stream, stats=False)
        # the depths are final: copy them out on a second stream while PageRank and colouring run
        bfs_done = torch.cuda.Event()
        bfs_done.record(stream)
        copy_stream.wait_event(bfs_done)
        with torch.cuda.stream(copy_stream):
            depths_h.copy_(depths, non_blocking=True)
        G.pagerank(ALPHA, EPS, rank_t, cfg=cfg_pr, stream=stream, stats=False)
        G.color(colors, cfg=cfg_gc, stream=stream, stats=False)
        rank_h.copy_(rank_t, non_blocking=True)
        colors_h.copy_(colors, non_blocking=True)
        torch.cuda.synchronize()
        G.close()

    step()
    steps = max(1, min(args.steps, 3))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    dt = max_over_ranks(time.perf_counter() - t0, world, "cuda") / steps
    h2d = 4 * (g.n + 1) + 4 * g.nnz + 4 * NSRC
    d2h = 4 * NSRC * g.n + 4 * g.n + 4 * g.n
    return {"value": round(world * work / dt / 1e9, 3), "unit": UNIT, "ms_per_step": round(dt * 1e3, 3),
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "note": "graph created from pinned host CSR (validation skipped: checked once before), results "
                    "copied back to pinned host memory (the BFS depths on a second stream, overlapped with "
                    "PageRank and colouring), all inside the timed region"}


# ------------------------------------------------------------------- batched-mix workload

BATCH_METRIC = "GTEPS (batched mix: 256 graphs x (4 BFS + 1 PageRank), one batched launch)"
BATCH_BFS = 4


def batched_workload(seed: int = 1):
    """128 RMAT graphs (scale 10..18) and 128 grids (side 64..1024), 10% of edges deleted each;
    per graph 4 BFS instances from seeded sources of nonzero degree and one PageRank."""
    graphs = [gg.materialise(spec) for spec in gg.batched_mix(seed=seed)]
    specs = []
    for gi, g in enumerate(graphs):
        for src in gg.sources(g, BATCH_BFS, seed=seed + gi):
            specs.append(("bfs", gi, int(src)))
        specs.append(("pagerank", gi, ALPHA, EPS))
    return graphs, specs


def batched_config(graphs, specs, extra=None):
    n = sum(g.n for g in graphs)
    nnz = sum(g.nnz for g in graphs)
    cfg = {"workload": "batched_mix_256g_bfs4_pr1", "graphs": "128 RMAT (scale U{10..18}, edge factor 16) + 128 "
           "grids (side U{64..1024}), 10% edge deletion, seed 1", "instances": len(specs),
           "bfs_instances": sum(1 for sp in specs if sp[0] == "bfs"), "n_total": n, "nnz_total": nnz,
           "alpha": ALPHA, "eps": EPS,
           "l2": f"inputs larger than L2: col is {nnz * 4 / 2**20:.0f} MiB in total vs 129 MiB L2 (no flush)"}
    if extra:
        cfg.update(extra)
    return cfg


def run_batched(args, rank: int, world: int):
    import torch

    import paper_2112_00132_gb300 as atos

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    atos.build() if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    atos.lib()
    graphs, specs = batched_workload()
    stream = torch.cuda.current_stream()
    Gs = [atos.Graph.from_csr(g) for g in graphs]
    # the batch's configuration: the autotuner's choice (worker, fetch, window, persistent vs
    # discrete, PageRank enqueue rule; an untimed sweep), unless fixed
    if args.no_tune:
        cfg, tune_ms = atos.queue_config(worker_size=args.worker, fetch_size=args.fetch), None
    else:
        cfg, tune_ms = atos.batch_autotune(Gs, specs, repeats=1, stream=stream)
    use_graph = cfg.strategy == atos.PERSISTENT  # discrete generations are driven by the host
    B = atos.Batch(Gs, specs, cfg)

    # warm-up (through the captured graph when persistent); the last one with statistics counts
    # the work
    for _ in range(max(args.warmup, 3)):
        B.run(stream=stream, graph=use_graph)
    _, per = B.stats(stream=stream)
    bfs_edges = pr_edges = pr_tasks = 0
    bfs_bytes = 0.0
    for (kind, gi, *rest), out, st in zip(specs, B.outputs, per):
        if st.status != 0:
            raise RuntimeError(f"batched instance {kind} on graph {gi} failed: {st.status}")
        g = graphs[gi]
        if kind == "bfs":
            deg = torch.from_numpy(np.diff(g.row_ptr).astype(np.int64)).cuda()
            comp = int(((out != 2**31 - 1).to(torch.int64) * deg).sum().item())  # directed entries
            bfs_edges += comp // 2
            bfs_bytes += 12.0 * g.n + 8.0 * comp
        else:
            pr_edges += st.edges
            pr_tasks += st.tasks
    work = bfs_edges + pr_edges

    l0 = atos.kernel_launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clocks:
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record(stream)
        for k in range(args.steps):
            B.run(stream=stream, graph=use_graph)
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
    launches = atos.kernel_launches() - l0
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    total_ms = max_over_ranks(evs[0].elapsed_time(evs[-1]), world, "cuda")
    if world > 1:
        torch.distributed.barrier()
    ms_step, value = replica_throughput(work, total_ms, args.steps, world)

    comparisons = {}
    if not args.no_compare:
        def timed(fn):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            fn()
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b)
        if use_graph:
            comparisons["batched_no_graph_ms"] = round(timed(lambda: B.run(stream=stream)), 3)
        outs = [(torch.empty((BATCH_BFS, g.n), dtype=torch.int32, device="cuda"),
                 torch.empty(g.n, dtype=torch.float32, device="cuda")) for g in graphs]
        srcs = [[sp[2] for sp in specs if sp[0] == "bfs" and sp[1] == gi] for gi in range(len(graphs))]

        def unbatched():
            for gi, G in enumerate(Gs):
                G.bfs(srcs[gi], outs[gi][0], cfg=cfg, stream=stream, stats=False)
                G.pagerank(ALPHA, EPS, outs[gi][1], cfg=cfg, stream=stream, stats=False)
        comparisons["per_graph_calls_ms"] = round(timed(unbatched), 3)
        del outs
        comparisons["batched_ms"] = round(statistics.mean(step_ms), 3)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    dom_bytes = bfs_bytes + 20.0 * pr_tasks + 8.0 * pr_edges
    dom_ms = statistics.mean(step_ms)
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    roofline = {"kernel": "batched_mixed_persistent", "bound": "hbm", "achieved": round(achieved, 1),
                "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback", "traffic": None,
                "algorithmic_bytes": dom_bytes, "launch_ms": round(dom_ms, 3)}
    result = {
        "metric": BATCH_METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32 (BFS) + f32 (PageRank)", "data": "synthetic",
        "config": batched_config(graphs, specs, {"window": B.window, "grid": B.grid, "worker": cfg.worker_size,
                                                 "fetch": cfg.fetch_size, "fetch_policy": cfg.fetch_policy,
                                                 "strategy": {0: "persistent", 1: "discrete"}.get(cfg.strategy),
                                                 "flags": cfg.flags, "cuda_graph": use_graph,
                                                 "autotuned": not args.no_tune, "autotune_best_ms": tune_ms,
                                                 "parallelism": f"replicas x{world}"}),
        "comparisons": comparisons, "roofline": roofline, "gpu_launches": launches,
        "breakdown": {"p50_ms": round(float(np.percentile(step_ms, 50)), 3),
                      "p99_ms": round(float(np.percentile(step_ms, 99)), 3),
                      "bfs_graph500_edges": bfs_edges, "pagerank_edge_pushes": pr_edges,
                      "pagerank_tasks": pr_tasks},
        "clocks": clocks.summary(),
    }
    B.close()
    for G in Gs:
        G.close()
    if not args.no_e2e:
        result["e2e"] = run_batched_e2e(args, graphs, specs, cfg, work, world)
    return result


def run_batched_e2e(args, graphs, specs, cfg, work, world):
    """The batched step through the public API from pinned host buffers: create the 256 graphs,
    build and run the batch, read every instance's output back, destroy everything."""
    import torch

    import paper_2112_00132_gb300 as atos
    stream = torch.cuda.current_stream()
    host = [(torch.from_numpy(g.row_ptr).pin_memory(), torch.from_numpy(g.col).pin_memory()) for g in graphs]
    outs_h = [torch.empty(graphs[sp[1]].n, dtype=torch.int32 if sp[0] == "bfs" else torch.float32).pin_memory()
              for sp in specs]

    def step():
        Gs = [atos.Graph(rp.numpy(), col.numpy(), skip_validation=True, stream=stream) for rp, col in host]
        with atos.Batch(Gs, specs, cfg) as B:
            B.run(stream=stream)
            for o_h, o in zip(outs_h, B.outputs):
                o_h.copy_(o, non_blocking=True)
            torch.cuda.synchronize()
        for G in Gs:
            G.close()

    step()
    steps = max(1, min(args.steps, 3))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    dt = max_over_ranks(time.perf_counter() - t0, world, "cuda") / steps
    h2d = sum(4 * (g.n + 1) + 4 * g.nnz for g in graphs)
    d2h = sum(4 * graphs[sp[1]].n for sp in specs)
    return {"value": round(world * work / dt / 1e9, 3), "unit": UNIT, "ms_per_step": round(dt * 1e3, 3),
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "note": "256 graphs created from pinned host CSR, batch built and run (no graph capture), every "
                    "instance's output copied back to pinned host memory, inside the timed region"}


BATCH_SAMPLE_STRIDE = 4


def cpu_baseline_batched(graphs, specs, stride=BATCH_SAMPLE_STRIDE):
    """Serial oracle on a bounded sample of the batched workload: the BFS instances and two
    power-iteration sweeps (nnz edge operations each) of every `stride`-th graph."""
    import oracle
    oracle.build()
    work = 0.0
    t0 = time.perf_counter()
    for kind, gi, *rest in specs:
        if gi % stride:
            continue
        g = graphs[gi]
        if kind == "bfs":
            d = oracle.bfs(g, rest[0])
            work += np.diff(g.row_ptr)[d != oracle.UNREACHED].sum() / 2
        else:
            oracle.pagerank_sweeps(g, ALPHA, 2)
            work += 2 * g.nnz
    dt = time.perf_counter() - t0
    return work, dt


def cpu_parallel_batched(graphs, specs):
    """The whole batched workload on every host core with the OpenMP baseline: each graph's BFS
    sources together (one serial search per thread) and its PageRank by Jacobi sweeps to the
    per-vertex epsilon.  Work counted as in the metric (component edges per BFS, nnz per sweep)."""
    try:
        from oracle import parallel
        parallel.build()
        threads = os.cpu_count() or 1
        by_graph = {}
        for kind, gi, *rest in specs:
            by_graph.setdefault(gi, []).append((kind, rest))
        work = 0.0
        t0 = time.perf_counter()
        for gi, items in by_graph.items():
            g = graphs[gi]
            srcs = [rest[0] for kind, rest in items if kind == "bfs"]
            if srcs:
                d, _ = parallel.bfs(g, srcs, nthreads=threads)
                deg = np.diff(g.row_ptr)
                work += sum(float(deg[row != np.iinfo(np.int32).max].sum()) / 2 for row in d)
            for kind, rest in items:
                if kind == "pagerank":
                    _, sweeps = parallel.pagerank(g, rest[0], rest[1], nthreads=threads)
                    work += sweeps * g.nnz
        dt = time.perf_counter() - t0
        return {"value": round(work / dt / 1e9, 4), "unit": UNIT, "cores": threads, "kind": "openmp",
                "sample": "the whole batch: every graph's BFS sources (one serial search per thread) and its "
                          "PageRank by FP64 Jacobi sweeps to the same per-vertex epsilon",
                "seconds": round(dt, 3)}
    except (OSError, RuntimeError, ValueError, subprocess.CalledProcessError) as e:
        return {"unavailable": f"OpenMP baseline: {type(e).__name__}: {e}"}


# --------------------------------------------------------------------------- CPU oracle arm

def oracle_sample(g, srcs, nbfs=1, sweeps=3, color=True, info=None):
    """Serial oracle on a bounded sample of the step; returns (work in the metric's units, seconds).
    `info` (a dict) receives the serial greedy colour count when the sample colours."""
    import oracle
    oracle.build()
    deg = np.diff(g.row_ptr)
    work = 0.0
    t0 = time.perf_counter()
    for s in srcs[:nbfs]:
        d = oracle.bfs(g, int(s))
        work += deg[d != oracle.UNREACHED].sum() / 2
    if sweeps:
        oracle.pagerank_sweeps(g, ALPHA, sweeps)
        work += sweeps * g.nnz
    if color:
        _, k = oracle.greedy_color(g)
        work += g.nnz
        if info is not None:
            info["serial_greedy_colors"] = k
    return work, time.perf_counter() - t0


def cpu_baseline(g, srcs):
    info = {}
    work, dt = oracle_sample(g, srcs, nbfs=2, sweeps=3, color=True, info=info)
    return {"value": round(work / dt / 1e9, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "serial C oracle, one thread: BFS from 2 of the 64 sources, 3 FP64 power-iteration "
                      "sweeps (nnz edge operations each), one greedy colouring (nnz entries)",
            "seconds": round(dt, 2), "host_cores": os.cpu_count(), **info}


def cpu_parallel(g, srcs):
    """The whole step on every host core with the OpenMP baseline (not the oracle): BFS from all
    sources, PageRank by Jacobi sweeps to the same per-vertex epsilon, speculative colouring.
    Work counted as in the metric (component edges per BFS, nnz per sweep, entries read by the
    colouring); `step_seconds` is the wall time of the three."""
    try:
        from oracle import parallel
        parallel.build()
        threads = os.cpu_count() or 1
        deg = np.diff(g.row_ptr)
        t0 = time.perf_counter()
        d, _ = parallel.bfs(g, srcs, nthreads=threads)
        t1 = time.perf_counter()
        _, sweeps = parallel.pagerank(g, ALPHA, EPS, nthreads=threads)
        t2 = time.perf_counter()
        _, k, rounds, gc_edges = parallel.color(g, nthreads=threads)
        t3 = time.perf_counter()
        bfs_edges = sum(float(deg[row != np.iinfo(np.int32).max].sum()) / 2 for row in d)
        work = bfs_edges + sweeps * g.nnz + gc_edges
        return {"value": round(work / (t3 - t0) / 1e9, 4), "unit": UNIT, "cores": threads, "kind": "openmp",
                "sample": f"the whole step: BFS from all {len(srcs)} sources (one serial search per thread), "
                          f"FP64 Jacobi PageRank until a sweep changes L1 by <= {EPS:g} n, speculative greedy "
                          "colouring in rounds",
                "step_seconds": round(t3 - t0, 3), "bfs_s": round(t1 - t0, 3), "pagerank_s": round(t2 - t1, 3),
                "color_s": round(t3 - t2, 3), "pagerank_sweeps": sweeps, "colors": k, "color_rounds": rounds}
    except (OSError, RuntimeError, ValueError, subprocess.CalledProcessError) as e:
        return {"unavailable": f"OpenMP baseline: {type(e).__name__}: {e}"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    if getattr(args, "workload", "rmat22") == "batched":
        return run_reference_batched(args, world)
    g, srcs = workload(args.scale)
    for _ in range(args.warmup):
        oracle_sample(g, srcs, nbfs=1, sweeps=1, color=False)
    works, times = [], []
    for _ in range(args.steps):
        w, dt = oracle_sample(g, srcs, nbfs=1, sweeps=2, color=True)
        works.append(w)
        times.append(dt)
    value = sum(works) / sum(times) / 1e9
    ms = 1e3 * sum(times) / len(times)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32 + f64", "data": "synthetic",
            "config": workload_config(g, args, {"strategy": "serial CPU oracle"}),
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "kind": "oracle", "cores": 1,
                             "sample": "per step: BFS from one of the 64 sources, 2 FP64 power-iteration sweeps, "
                                       "one greedy colouring"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_batched(args, world):
    graphs, specs = batched_workload()
    for _ in range(args.warmup):
        cpu_baseline_batched(graphs, specs, stride=64)
    works, times = [], []
    for _ in range(args.steps):
        w, dt = cpu_baseline_batched(graphs, specs)
        works.append(w)
        times.append(dt)
    value = sum(works) / sum(times) / 1e9
    sample = "per step: the 4 BFS instances and 2 FP64 power-iteration sweeps of every 4th graph (64 graphs)"
    return {"impl": "reference", "metric": BATCH_METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / len(times), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32 + f64",
            "data": "synthetic", "config": batched_config(graphs, specs, {"strategy": "serial CPU oracle"}),
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "kind": "oracle", "cores": 1, "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    if args.study == "color-ids":
        res = run_color_ids_study(args) if rank == 0 else None
    elif args.impl == "reference":
        res = run_reference(args, rank, world)
    elif args.workload == "batched":
        res = run_batched(args, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            graphs, specs = batched_workload()
            w, dt = cpu_baseline_batched(graphs, specs)
            res["cpu_baseline"] = {"value": round(w / dt / 1e9, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": "serial C oracle, one thread: the 4 BFS instances and 2 FP64 "
                                             "power-iteration sweeps of every 4th graph (64 graphs)",
                                   "seconds": round(dt, 2), "host_cores": os.cpu_count()}
            res["cpu_parallel"] = cpu_parallel_batched(graphs, specs)
    else:
        res = run_atos(args, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            g, srcs = workload(args.scale)
            res["cpu_baseline"] = cpu_baseline(g, srcs)
            res["breakdown"]["colors_serial_greedy"] = res["cpu_baseline"].get("serial_greedy_colors")
            res["cpu_parallel"] = cpu_parallel(g, srcs)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
