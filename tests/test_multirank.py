"""Multi-rank (weak-scaling replica) logic of bench.py on CPU with gloo, world size 2.

Compressions are independent jobs, so N GPUs run N replicas with no data-path
collective; the only cross-rank operations are the timing barrier and the
max-over-ranks reduction, tested here without a GPU.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = 1.0 + rank                    # rank 1 is the slow one
        tmax = bench.reduce_max(seconds, world)
        value = bench.weak_value(4, world, tmax)
        pts0, *_ = bench.make_inputs(bench.WORKLOADS["laplace2d_n16384"], rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, float(pts0[0, 0]))
        q.put((rank, tmax, value, gathered))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_ranks_take_the_max_time_and_distinct_inputs():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, tmax, value, gathered in out:
        assert tmax == 2.0                      # max over ranks
        assert value == 4 * 2 / 2.0             # all ranks' work over the slowest time
        assert gathered[0] != gathered[1]       # replicas draw their own inputs


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        cpu_sample_boxes = 1
        warmup = 0
        steps = 1
        workload = "laplace2d_n16384"
    assert bench.run_reference(Args, dict(bench.WORKLOADS["laplace2d_n16384"])) is None
