"""Request-serving loop over resident graphs (continuous batching on the GPU).

Requests arrive as a Poisson process (seeded; exponential inter-arrival times), each a BFS (from a
random source of nonzero degree), a PageRank or a colouring on a graph drawn uniformly from the
resident set, in the proportions of ``mix``.  The loop admits every arrived request it can (the
server refuses while no slot or arena memory is free), runs one server epoch (a persistent launch
bounded by ``slice_ns`` over every admitted request), and records each completion's latency =
completion time - arrival time.  Requests that arrive during the warm-up are served but not
counted.

Admission keeps two FIFO queues: requests on graphs of more than ``large_n`` vertices, of which at
most ``max_large`` are admitted at a time, and the rest.  Without the split, slots fill up with
the long requests under overload (each finishes late, so the slots they hold turn over slowly)
and the completion rate falls below what the GPU sustains.

Usage: python -m paper_2112_00132_gb300.serve [--rate 2000] [--duration 10] [--warmup 1]
       [--graphs small|config]   (``config``: 64 graphs of the batched mix plus RMAT 23)
       [--rates 100,200,400]     (a sweep: one JSON line per offered rate, graphs uploaded once)
Prints one JSON line per rate with p50 / p99 latency, achieved rate and throughput.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import graphgen as gg  # noqa: E402

from paper_2112_00132_gb300 import _binding as abi  # noqa: E402

STREAM_ARRIVALS = gg.STREAM_ARRIVALS


def make_arrivals(rate: float, duration: float, mix, ngraphs: int, seed: int = 1):
    """[(time, kind, graph)] for a Poisson process of `rate` per second over `duration` seconds."""
    out = []
    t = 0.0
    i = 0
    kinds = ("bfs", "pagerank", "color")
    cum = np.cumsum(mix) / np.sum(mix)
    while True:
        u = (gg.stream_u64(seed, STREAM_ARRIVALS, 3 * i) >> 11) / 9007199254740992.0
        t += -math.log(1.0 - u) / rate
        if t >= duration:
            break
        uk = (gg.stream_u64(seed, STREAM_ARRIVALS, 3 * i + 1) >> 11) / 9007199254740992.0
        ug = (gg.stream_u64(seed, STREAM_ARRIVALS, 3 * i + 2) >> 11) / 9007199254740992.0
        out.append((t, kinds[int(np.searchsorted(cum, uk, side="right"))], min(int(ug * ngraphs), ngraphs - 1)))
        i += 1
    return out


def serve(csrs, rate=2000.0, duration=10.0, warmup=1.0, mix=(0.6, 0.3, 0.1), slice_ns=1_000_000, max_slots=64,
          budget_bytes=None, alpha=0.85, eps=1e-9, seed=1, drain_s=30.0, keep=0, cfg=None, graphs=None,
          large_n=1 << 21, max_large=1, server_factory=None):
    """Runs the serving loop; returns a summary dict (and up to `keep` finished requests with their
    outputs under "kept", for checking).  `graphs`: resident abi.Graph objects of `csrs` to reuse
    (created here, and closed at the end, when None).  `server_factory(graphs, max_slots,
    budget_bytes, cfg)` builds the server (default: abi.Server); the loop only calls its submit,
    step, poll, info and close."""
    own_graphs = graphs is None
    if own_graphs:
        graphs = [abi.Graph.from_csr(g) for g in csrs]
    sources = [gg.sources(g, 4096, seed=seed + 11 * k) if g.nnz else np.zeros(1, np.int32)
               for k, g in enumerate(csrs)]
    if budget_bytes is None:
        import torch
        free, _ = torch.cuda.mem_get_info()
        budget_bytes = int(min(free * 0.5, 64 << 30))
    if cfg is None:  # PageRank and colouring on the graphs' spread-id copies (faster on every graph measured)
        cfg = abi.queue_config(flags=abi.FLAG_SPREAD_IDS)
    if server_factory is None:
        server = abi.Server(graphs, max_slots=max_slots, budget_bytes=budget_bytes, cfg=cfg)
    else:
        server = server_factory(graphs, max_slots, budget_bytes, cfg)
    arrivals = make_arrivals(rate, duration, mix, len(graphs), seed)
    backlog, backlog_large = [], []
    large_active = 0
    is_large = [g.n > large_n for g in csrs]
    meta = {}
    lat = []
    kept = []
    edges_done = 0
    completed = 0
    per_kind = {"bfs": [], "pagerank": [], "color": []}
    t0 = time.perf_counter()
    nxt = 0
    steps = 0
    while True:
        now = time.perf_counter() - t0
        while nxt < len(arrivals) and arrivals[nxt][0] <= now:
            (backlog_large if is_large[arrivals[nxt][2]] else backlog).append((nxt,) + arrivals[nxt])
            nxt += 1
        # admit in arrival order while the server accepts: the large-graph queue first, up to
        # max_large of them in flight, then the others
        for queue, large in ((backlog_large, True), (backlog, False)):
            while queue and (not large or large_active < max_large):
                idx, t_arr, kind, gi = queue[0]
                src = int(sources[gi][idx % len(sources[gi])])
                got = server.submit(kind, gi, source=src, alpha=alpha, eps=eps)
                if got is None:
                    break
                meta[got[0]] = (t_arr, kind, gi, src)
                large_active += large
                queue.pop(0)
        left = server.step(slice_ns)
        steps += 1
        t_done = time.perf_counter() - t0
        for c in server.poll():
            t_arr, kind, gi, src = meta.pop(c["id"])
            large_active -= is_large[gi]
            completed += 1
            if c["status"] != 0:
                continue
            if t_arr >= warmup:
                lat.append(t_done - t_arr)
                per_kind[kind].append(t_done - t_arr)
                edges_done += c["edges"]
            if len(kept) < keep:
                kept.append({"kind": kind, "graph": gi, "source": src, "out": c["out"], "error_bound": c["error_bound"]})
        now = time.perf_counter() - t0
        if nxt >= len(arrivals) and not backlog and not backlog_large and left == 0:
            break
        if now > duration + drain_s:
            break
        if left == 0 and not backlog and not backlog_large and nxt < len(arrivals):
            time.sleep(max(0.0, min(arrivals[nxt][0] - now, 0.001)))
    wall = time.perf_counter() - t0
    window = max(1e-9, min(wall, duration) - warmup)
    measured = [a for a in arrivals if a[0] >= warmup]
    lat_ms = np.array(lat) * 1e3
    info = server.info()
    server.close()
    if own_graphs:
        for g in graphs:
            g.close()
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None  # noqa: E731
    achieved = len(lat) / window
    offered = len(measured) / max(1e-9, duration - warmup)
    res = {
        "offered_rps": round(offered, 1), "achieved_rps": round(achieved, 1),
        "sustainable": bool(len(lat) >= 0.95 * len(measured) and wall <= duration + 1.0),
        "requests": len(arrivals), "completed": completed, "unfinished": len(meta) + len(backlog) + len(backlog_large),
        "p50_ms": pct(lat_ms, 50), "p99_ms": pct(lat_ms, 99), "mean_ms": float(lat_ms.mean()) if len(lat) else None,
        "p50_ms_by_kind": {k: pct(np.array(v) * 1e3, 50) for k, v in per_kind.items()},
        "p99_ms_by_kind": {k: pct(np.array(v) * 1e3, 99) for k, v in per_kind.items()},
        "gteps": round(edges_done / window / 1e9, 3),
        "gteps_unit": "neighbour entries read by task bodies per second (directed, includes overwork)",
        "epochs": info["epochs"], "steps": steps, "slice_ms": slice_ns / 1e6, "wall_s": round(wall, 2),
        "graphs": len(csrs), "max_slots": max_slots, "arena_bytes": budget_bytes,
        "admission": f"two FIFO queues; at most {max_large} requests on graphs of > {large_n} vertices in flight",
        "config": {"worker": cfg.worker_size, "fetch": cfg.fetch_size, "flags": cfg.flags},
    }
    if keep:
        res["kept"] = kept
    return res


def config_graphs(seed: int = 1):
    """The serving workload's resident set: 64 graphs drawn as in the batched mix (RMAT scale
    10..18 or grid side 64..1024, 10% edge deletion) plus one RMAT scale 23."""
    mix = gg.batched_mix(seed=seed)
    pick = [mix[int((gg.stream_u64(seed, STREAM_ARRIVALS + 1, i) >> 11) * len(mix) / 9007199254740992.0)]
            for i in range(64)]
    out = [gg.materialise(spec) for spec in pick]
    out.append(gg.rmat(23, 16, seed=seed))
    return out


def small_graphs(seed: int = 1):
    return [gg.rmat(12, 16, seed=seed), gg.grid(120, 90, delete_frac=0.1, seed=seed), gg.rmat(14, 16, seed=seed + 1),
            gg.grid(300, 300, delete_frac=0.1, seed=seed + 2)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--warmup", type=float, default=1.0)
    ap.add_argument("--slice-ms", type=float, default=1.0)
    ap.add_argument("--graphs", default="config", choices=["config", "small"])
    ap.add_argument("--max-slots", type=int, default=64)
    ap.add_argument("--drain", type=float, default=30.0, help="seconds allowed after the last arrival")
    ap.add_argument("--rates", default="", help="comma-separated offered rates (a sweep); overrides --rate")
    ap.add_argument("--max-large", type=int, default=1, help="requests on large graphs in flight at most")
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    abi.lib()
    csrs = config_graphs() if args.graphs == "config" else small_graphs()
    graphs = [abi.Graph.from_csr(g) for g in csrs]
    rates = [float(r) for r in args.rates.split(",") if r] or [args.rate]
    for rate in rates:
        res = serve(csrs, rate=rate, duration=args.duration, warmup=args.warmup, slice_ns=int(args.slice_ms * 1e6),
                    max_slots=args.max_slots, drain_s=args.drain, graphs=graphs, max_large=args.max_large)
        res["workload"] = ("64 graphs of the batched mix + RMAT 23" if args.graphs == "config" else "4 small graphs")
        res["mix"] = "BFS 60% / PageRank 30% / colouring 10%"
        print(json.dumps(res), flush=True)
    for g in graphs:
        g.close()


if __name__ == "__main__":
    main()
