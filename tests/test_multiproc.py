"""The N-GPU path of the benchmark, on CPU: two gloo ranks run the same
whole-job aggregation bench.py uses under torchrun (step time = MAX over
ranks, work = SUM over ranks; trials are sharded, nothing else is
exchanged).  No GPU is used."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def allreduce(x, op):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=op)
        return t.item()

    ops = {"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}
    # rank r: its own FOS step of 1000 + r trials with 5000 active nodes each,
    # 10 steps taking (20 + 5 r) ms in total
    out = bench.aggregate(20.0 + 5 * rank, 10, 5000 * (1000 + rank), 1000 + rank, 100_000,
                          allreduce, ops)
    assert bench.dist_env() == (rank, world, rank)
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ms = (20.0 + 5) / 10  # the slower rank
    nodes = 5000 * 1000 + 5000 * 1001
    for r in range(world):
        out = res[r]
        assert out["ms_per_step"] == pytest.approx(ms)
        assert out["node_row_evals_per_s"] == pytest.approx(nodes * 100_000 / (ms * 1e-3))
        assert out["trial_evals_per_s"] == pytest.approx(2001 / (ms * 1e-3))
