"""The benchmark's multi-GPU path (independent replicas, no collective on the
data path) as two gloo ranks on the CPU: each rank takes different frames, the
job's time is the slowest rank's, the throughput counts every rank's frames."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [120.0, 150.0][rank]                      # rank 1 is the slower replica
        t = bench.max_over_ranks(ms, world)
        out[rank] = (t, bench.job_throughput(16, 20, world, t), bench.replica_seeds(rank, 16))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        ctx = mp.get_context("spawn")
        port = _free_port()                                    # both ranks rendezvous here
        ps = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0                     # max over ranks
    assert res[0][1] == pytest.approx(16 * 20 * 2 / 0.150)     # all frames / slowest time
    assert set(res[0][2]).isdisjoint(res[1][2])                # different frames per rank
    assert bench.max_over_ranks(42.0, 1) == 42.0               # one GPU: no collective
