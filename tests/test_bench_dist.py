"""The multi-replica path of bench.py (one independent replica per rank, no
data-path collective): max-over-ranks timing and the whole-job rate, run as two
gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(('127.0.0.1', 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    import bench
    # replicas finish at different times; the job takes the slowest one
    local = [0.8, 1.25][rank]
    t = bench.max_over_ranks(local, world, 'cpu')
    out[rank] = (t, bench.job_rate(1000, 10, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 1.25
    # 2 replicas x 1000 cells x 10 steps in 1.25 s
    assert res[0][1] == pytest.approx(2 * 1000 * 10 / 1.25 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, 1, 'cpu') == 3.0
    assert bench.job_rate(4194304, 40, 1, 0.1) == pytest.approx(4194304 * 40 / 0.1 / 1e6)
