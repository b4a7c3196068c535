"""The multi-process path of bench.py (one process per GPU, replicas with no
collective on the data path) exercised with two gloo ranks on the CPU:
disjoint instance seeds per rank, max-over-ranks timing, the whole-job
aggregate, and the reference arm running on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    batch = 5
    seeds = list(range(bench.rank_seed0(batch, rank), bench.rank_seed0(batch, rank) + batch))
    # rank r "took" 100 + 10 r ms; every rank must see the slowest
    ms = bench.max_over_ranks(100.0 + 10.0 * rank, world, "cpu")
    rate = bench.aggregate_rate(batch, world, 3, ms / 1e3)

    class A:
        steps, warmup = 1, 0
    ref = bench.run_reference(A(), rank, world) if rank != 0 else None
    out[rank] = (seeds, ms, rate, ref)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    s0, s1 = set(res[0][0]), set(res[1][0])
    assert len(s0) == len(s1) == 5 and not (s0 & s1)          # disjoint instances
    assert res[0][1] == res[1][1] == 110.0                      # max over ranks
    assert res[0][2] == pytest.approx(5 * 2 * 3 / 0.110)       # whole-job aggregate
    assert res[1][3] == 0                                       # reference arm: rank 1 does no work
