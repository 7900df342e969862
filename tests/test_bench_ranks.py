"""The multi-rank bookkeeping of ``bench.py --gpus N`` (N independent replicas,
no data-path collective): the job's step time is the slowest rank's, and the
whole-job rate counts every replica.  Two gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [12.5, 17.0][rank]
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (ms, bench.job_rate(ms, world))
    finally:
        dist.destroy_process_group()


def test_replicas_timed_to_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    for r in range(world):
        ms, rate = res[r]
        assert ms == 17.0
        assert rate == pytest.approx(2 * 1e3 / 17.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(4.0, 1) == 250.0
