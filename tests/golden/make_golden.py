"""Writes the stored expected values under tests/golden/ from the CPU oracle alone.

Only ``oracle`` and ``graphgen`` are called here; nothing comes from the CUDA path.  The paper
prints no worked example with values (its figures are runtimes and workload ratios on datasets
that are not available), so every stored value is an oracle value for a seeded synthetic graph,
kept to catch regressions of the oracle itself.

Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402


def summary(g, sources):
    out = {"graph": g.name, "n": g.n, "nnz": g.nnz, "bfs": {}}
    for s in sources:
        d = oracle.bfs(g, int(s))
        reached = d[d != oracle.UNREACHED]
        out["bfs"][str(int(s))] = {"reached": int(reached.size),
                                   "depth_histogram": np.bincount(reached).tolist()}
    x, sweeps, _ = oracle.pagerank(g, 0.85)
    q = x / x.sum()
    top = np.argsort(-q, kind="stable")[:8]
    out["pagerank"] = {"alpha": 0.85, "sum_unnormalised": float(x.sum()),
                       "top": [[int(v), float(q[v])] for v in top]}
    c, k = oracle.greedy_color(g)
    out["greedy_colors"] = k
    return out


def main():
    cases = {
        "rmat12_s1.json": (gg.rmat(12, 16, seed=1), [0, 1, 2, 77]),
        "grid64_del10_s1.json": (gg.grid(64, 64, delete_frac=0.1, seed=1), [0, 2080]),
    }
    for fname, (g, srcs) in cases.items():
        with open(os.path.join(HERE, fname), "w") as f:
            json.dump(summary(g, srcs), f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main()
