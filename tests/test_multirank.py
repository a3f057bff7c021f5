"""Multi-rank (replica) host logic of bench.py on CPU: two gloo ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow replica
        got = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        thr = bench.job_throughput(world, 1000, got / 1e3)
        out[rank] = (got, thr)
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (15.0, 2 * 1000 / 0.015)


def test_single_process_has_no_reduction():
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.job_throughput(1, 10, 2.0) == 5.0
