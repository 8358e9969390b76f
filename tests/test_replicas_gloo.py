"""The N > 1 path of bench.py on CPU: two gloo ranks, no GPU.

The solve does not shard (every rank factors and solves its own problem), so
the only cross-rank step is the timing: the job's time is the slowest
replica's (all-reduce MAX) and the whole-job rate counts every rank's units.
These ranks report different local times and check that both see the
maximum and the same aggregate.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local = [0.75, 1.25][rank]          # seconds for `steps` steps on this rank
        sec = bench.max_over_ranks(local)
        val = bench.whole_job_value(1000.0, 5, sec, world)
        out[rank] = (sec, val)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_the_sum_of_units():
    world = 2
    with mp.get_context("spawn").Manager() as m:   # no fork of this threaded process
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for sec, val in res.values():
        assert sec == 1.25
        assert val == pytest.approx(2 * 1000.0 * 5 / 1.25, rel=1e-15)


def test_single_process_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(0.5) == 0.5
    assert bench.whole_job_value(10.0, 4, 2.0, 1) == 20.0
