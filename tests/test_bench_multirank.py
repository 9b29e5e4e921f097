"""bench.py's multi-rank aggregation on CPU with the gloo backend (world size 2):
ranks run independent replicas, the whole-job rate is the sum of the ranks'
units over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sec = [2.0, 5.0][rank]
    units = [100.0, 300.0][rank]
    rate, tmax = bench.whole_job_rate(sec, units, dist, "cpu")
    out[rank] = (rate, tmax)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        rate, tmax = out[r]
        assert tmax == 5.0
        assert abs(rate - 400.0 / 5.0) < 1e-12


def test_whole_job_rate_single_process():
    import bench
    rate, t = bench.whole_job_rate(4.0, 10.0, None)
    assert rate == 2.5 and t == 4.0
