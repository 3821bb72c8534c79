"""The benchmark's JSON line (CPU only): the oracle arm (``--impl reference``) on a small graph
prints one line with every key of the contract, and the GPU arm's helpers aggregate as stated."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--scale", "10", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["data"] == "synthetic"
    assert d["config"]["workload"] == "rmat10_bfs64_pagerank_color"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_recorded_traffic_lookup(tmp_path):
    """roofline.traffic: the entry for the run's PageRank shape, and only while the kernel sources
    hash to the recorded value."""
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "csrc"
    src.mkdir()
    for f in bench.TRAFFIC_SOURCES:
        (src / f).write_text(f"// {f}\nint x_{f.replace('.', '_')} = 1;\n")
    rec = tmp_path / "traffic.txt"
    rec.write_text("# header\nentry: 512 256 1 8 4 62810000000\nentry: 1024 1024 2 16 4 67650000000\n"
                   f"kernel_code_sha256: {bench.kernel_sources_digest(str(src))}\n")

    class Cfg:
        worker_size, fetch_size, fetch_policy, check_size, flags = 512, 256, 1, 8, 4
    assert bench.recorded_traffic(Cfg, path=str(rec), src_dir=str(src)) == 62810000000.0
    Cfg.check_size = 16
    assert bench.recorded_traffic(Cfg, path=str(rec), src_dir=str(src)) is None  # no such shape
    Cfg.check_size = 8
    (src / "pagerank.cuh").write_text("/* a comment\n   edited */ int x_pagerank_cuh   =  1;  // and here\n")
    assert bench.recorded_traffic(Cfg, path=str(rec), src_dir=str(src)) == 62810000000.0  # comments only
    (src / "pagerank.cuh").write_text("int x_pagerank_cuh = 2;\n")
    assert bench.recorded_traffic(Cfg, path=str(rec), src_dir=str(src)) is None  # code changed


def test_cpu_parallel_leg_shape():
    """The OpenMP comparison leg: the whole step on every host core, labelled as such."""
    import bench
    g, srcs = bench.workload(12)
    r = bench.cpu_parallel(g, srcs)
    assert r["kind"] == "openmp" and r["unit"] == bench.UNIT and r["cores"] >= 1
    assert r["value"] > 0 and r["step_seconds"] > 0 and r["pagerank_sweeps"] > 0 and r["colors"] >= 2


def test_cpu_parallel_batched_leg():
    """The OpenMP leg of the batched workload on a small mix: every graph's sources and PageRank."""
    import bench
    import graphgen as gg
    graphs = [gg.rmat(10, 8, seed=3), gg.grid(40, 30, delete_frac=0.1, seed=2)]
    specs = []
    for gi, g in enumerate(graphs):
        specs += [("bfs", gi, int(s)) for s in gg.sources(g, 4, seed=gi + 1)]
        specs.append(("pagerank", gi, 0.85, 1e-9))
    r = bench.cpu_parallel_batched(graphs, specs)
    assert r["kind"] == "openmp" and r["value"] > 0 and r["seconds"] > 0 and r["cores"] >= 1
