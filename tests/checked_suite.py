"""Parity cases run on the bounds-checked library (libatos_checked.so, built with ATOS_CHECKED).

A helper, not a test module: tests/test_gpu_checked.py runs it in a subprocess, so the process
loads the checked library instead of libatos.so, and reads the JSON line it prints.  Every case
of the small-graph suite must pass with no violation recorded (a violation would make the call
return ATOS_ERR_BOUNDS).  A planted out-of-range column index, which the host check is told to
skip, must be caught by the device checks of the CTA persistent worker and of the BSP advance.

Usage: python tests/checked_suite.py <path of libatos_checked.so>
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import paper_2112_00132_gb300._binding as B  # noqa: E402

B.LIB_PATH = sys.argv[1]

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402
import paper_2112_00132_gb300 as atos  # noqa: E402
from gpu_common import ALPHA, EPS, PR_L1_TOL, bfs_sources, configs, small_graphs, thread_worker_configs  # noqa: E402


def main():
    import torch
    torch.cuda.set_device(0)
    assert os.path.samefile(B.LIB_PATH, sys.argv[1])
    atos.lib()
    runs, failures = 0, []

    def fail(what):
        failures.append(what)

    graphs = dict(small_graphs())
    graphs["rmat14"] = gg.rmat(14, 16, seed=5)
    graphs["star12000"] = gg.star(12000)  # a row long enough to be split into segment tasks
    for gname, g in graphs.items():
        srcs = bfs_sources(g)
        bfs_ref = np.stack([oracle.bfs(g, s) for s in srcs])
        x, _, _ = oracle.pagerank(g, ALPHA)
        pr_ref = x / x.sum()
        greedy, kg = oracle.greedy_color(g)
        with atos.Graph.from_csr(g) as G:
            shapes = {**configs(atos), **thread_worker_configs(atos)}
            for cname, cfg in shapes.items():
                base = cfg.flags
                try:
                    for flags in (0, atos.FLAG_BFS_EXPAND_ONCE, atos.FLAG_BFS_EXPAND_ONCE | atos.FLAG_BFS_SPLIT_ROWS):
                        cfg.flags = base | flags
                        d, st = G.bfs(srcs, cfg=cfg)
                        runs += 1
                        if not np.array_equal(d.cpu().numpy(), bfs_ref):
                            fail(f"bfs {gname}/{cname}/{flags}")
                    for flags in (0, atos.FLAG_SPREAD_IDS, atos.FLAG_PR_CROSSING):
                        cfg.flags = base | flags
                        r, st = G.pagerank(ALPHA, EPS, cfg=cfg)
                        runs += 1
                        if np.abs(r.cpu().numpy().astype(np.float64) - pr_ref).sum() > PR_L1_TOL:
                            fail(f"pagerank {gname}/{cname}/{flags}")
                    for flags in (0, atos.FLAG_SPREAD_IDS, atos.FLAG_GC_DEPENDENCY):
                        cfg.flags = base | flags
                        c, k, st = G.color(cfg=cfg)
                        runs += 1
                        c = c.cpu().numpy()
                        if oracle.check_coloring(g, c)[0] != 0:
                            fail(f"color {gname}/{cname}/{flags}")
                        if flags == atos.FLAG_GC_DEPENDENCY and not cname.startswith("bsp") and \
                                not np.array_equal(c, greedy):
                            fail(f"color dependency {gname}/{cname}")
                except atos.AtosError as e:
                    fail(f"{gname}/{cname}: {e}")
    # a mixed batch, CTA and thread workers
    gs = [gg.rmat(11, 16, seed=2), gg.grid(60, 45, delete_frac=0.1, seed=4)]
    Gs = [atos.Graph.from_csr(x) for x in gs]
    specs = [("bfs", 0, 0), ("pagerank", 1), ("color", 0), ("bfs", 1, 7), ("pagerank", 0)]
    for cfg in (atos.queue_config(), atos.queue_config(worker_size=1, fetch_size=32)):
        try:
            with atos.Batch(Gs, specs, cfg) as b:
                b.run()
                _, per = b.stats()
                runs += 1
                if any(st.status for st in per):
                    fail(f"batch worker {cfg.worker_size}")
        except atos.AtosError as e:
            fail(f"batch worker {cfg.worker_size}: {e}")
    for G in Gs:
        G.close()
    # planted: vertex 0's first neighbour out of range, host validation skipped
    g = gg.grid(30, 30, seed=1)
    col = g.col.copy()
    col[g.row_ptr[0]] = g.n + 5
    planted = {}
    for name, cfg in (("persistent_cta", atos.queue_config()), ("bsp", atos.queue_config("bsp"))):
        with atos.Graph(g.row_ptr, col, skip_validation=True) as G:
            try:
                G.bfs([0], cfg=cfg)
                planted[name] = "not caught"
            except atos.AtosError as e:
                planted[name] = "caught" if e.status == atos.abi.ERR_BOUNDS else f"status {e.status}"
                if name == "persistent_cta":
                    planted["persistent_cta_site"] = G.queue_state(1)[1]
    ok = not failures and all(v == "caught" for k, v in planted.items() if not k.endswith("_site")) and \
        planted.get("persistent_cta_site") == 103
    print(json.dumps({"runs": runs, "failures": failures[:20], "planted": planted, "ok": ok}), flush=True)
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
