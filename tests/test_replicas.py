"""Multi-process (gloo, world size 2, CPU) checks of the benchmark's replica path: with N > 1 every
rank runs an independent replica of the single-GPU step (the graph algorithms do not shard), the
timed region's length is the maximum over ranks, whole-job throughput counts every replica's work,
and the oracle arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # per-rank timed-region lengths differ; every rank must see the slowest one
        ms = [120.0, 180.0][rank]
        total = bench.max_over_ranks(ms, world, "cpu")
        ms_step, value = bench.replica_throughput(3.0e9, total, 3, world)
        dist.barrier()

        class A:  # the arguments the oracle arm reads
            scale, steps, warmup = 8, 1, 0
        ref = bench.run_reference(A, rank, world)
        out.put((rank, total, ms_step, value, ref is None, None if ref is None else ref["n_gpus"]))
    finally:
        dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r = q.get(timeout=240)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        _, total, ms_step, value, ref_none, ngpu = res[r]
        assert total == 180.0
        assert ms_step == pytest.approx(60.0)
        # two replicas x 3e9 edges per step in 60 ms
        assert value == pytest.approx(2 * 3.0e9 / 0.060 / 1e9)
    assert res[1][4] and not res[0][4]
    assert res[0][5] == world


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.5, 1, "cpu") == 42.5
    ms_step, value = bench.replica_throughput(1.0e9, 200.0, 2, 1)
    assert ms_step == 100.0 and value == pytest.approx(10.0)
