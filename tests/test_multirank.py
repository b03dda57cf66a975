"""The N > 1 path of bench.py (independent replicas, one per rank): the
cross-rank combination -- slowest rank's time, particle-steps summed over
ranks -- run as two gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip('torch')
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(('127.0.0.1', 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group('gloo', rank=rank, world_size=world)
    import bench
    ms = [10.0, 12.5][rank]
    n = [24500, 24600][rank]
    total, value = bench.combine_ranks(ms, n, 100, world, 'cpu')
    out[rank] = (total, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_combination():
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method='spawn', join=True)
        res = dict(out)
    for r in (0, 1):
        total, value = res[r]
        assert total == 12.5
        assert value == pytest.approx((24500 + 24600) * 100 / 12.5e-3)


def test_single_rank_is_plain_throughput():
    import bench
    total, value = bench.combine_ranks(20.0, 1000, 10, 1, 'cpu')
    assert total == 20.0 and value == pytest.approx(1000 * 10 / 0.02)
