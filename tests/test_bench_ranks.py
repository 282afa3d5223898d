"""Multi-rank (replica) path of bench.py on CPU: world size 2 over gloo on 127.0.0.1.

Each rank times its own replica; the whole-job figure uses the slowest rank (MAX of the timed
totals) and counts every rank's stage solves."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip('torch')
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group('gloo', rank=rank, world_size=world)
    total, e2e = bench.aggregate_ranks(100.0 + 50.0 * rank, 20.0 - rank, world, 'cpu')
    out[rank] = (total, e2e, bench.job_rate(world, 3, 10, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    world = 2
    ctx = mp.get_context('spawn')
    with ctx.Manager() as man:
        out = man.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method='spawn', join=True)
        res = dict(out)
    for rank in range(world):
        total, e2e, rate = res[rank]
        assert total == 150.0 and e2e == 20.0
        assert rate == pytest.approx(2 * 3 * 10 / 0.150)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(12.5, 3.0, 1, 'cpu') == (12.5, 3.0)
    assert bench.job_rate(1, 3, 4, 1000.0) == pytest.approx(12.0)
