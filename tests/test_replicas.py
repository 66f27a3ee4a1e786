"""bench.py under torchrun runs one independent replica per GPU (a single
graph does not shard: pointer jumping crosses any partition).  The only
exchange between ranks is the timing reduction: the job takes as long as its
slowest rank, and its rate counts every rank's units.  Checked here with two
gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [40.0, 50.0][rank]          # the second rank is the slower one
    rate, job_ms = bench.job_rate(1000, 10, local_ms, world, "cpu")
    out[rank] = (rate, job_ms)
    dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_and_counts_all_units():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        rate, job_ms = res[rank]
        assert job_ms == 50.0
        assert rate == pytest.approx(2 * 10 * 1000 / 0.050)


def test_job_rate_on_one_rank_needs_no_process_group():
    import bench
    rate, job_ms = bench.job_rate(5, 4, 20.0, 1, "cpu")
    assert job_ms == 20.0 and rate == pytest.approx(5 * 4 / 0.020)
