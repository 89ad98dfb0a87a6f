"""Host logic of the benchmark's N-GPU path, run as world_size-2 gloo process groups on the CPU.

With more than one GPU every rank runs its own replica of the workload (the sweep has no exchange
step to shard), so the only cross-rank logic is reading the rank layout from the environment and
taking the slowest rank's step time for the whole-job rate.  No GPU is touched here.
"""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        ms = bench.max_over_ranks(1.5 + 2.0 * rank, "cpu")   # rank 1 is the slow one
        out[rank] = (r, w, local, ms, bench.job_rate(ms, w))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank in range(world):
        r, w, local, ms, rate = res[rank]
        assert (r, w, local) == (rank, world, rank)
        assert ms == 3.5                                   # both ranks see the slowest rank's time
        assert rate == pytest.approx(world * 1000.0 / 3.5)  # two replicas per 3.5 ms


def test_single_process_defaults():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    saved = {k: os.environ.pop(k) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_env() == (0, 1, 0)
        assert bench.job_rate(0.5, 1) == pytest.approx(2000.0)
    finally:
        os.environ.update(saved)
