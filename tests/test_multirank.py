"""The multi-rank path of bench.py (N replicas, one per GPU) on CPU ranks:
world_size 2 over gloo, 127.0.0.1.  The timed region is the slowest rank's
and the whole-job value counts every rank's units."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from bench import job_throughput
    local_ms = [120.0, 300.0][rank]   # the second rank is slower
    total_ms, value = job_throughput(local_ms, 1000, world)
    out[rank] = (total_ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_throughput_uses_the_slowest_rank():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    total_ms, value = res[0]
    assert total_ms == 300.0
    assert value == pytest.approx(2 * 1000 / 0.3)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    from bench import job_throughput
    assert job_throughput(250.0, 500, 1) == (250.0, 2000.0)
