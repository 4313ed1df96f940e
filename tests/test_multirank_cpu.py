"""The benchmark's multi-rank logic on CPU with two gloo ranks: the timed region
is the slowest rank's, and the whole-job throughput counts every rank's solves
(weak scaling: each rank solves its own replica; no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank                      # rank 1 is the slow one
    slowest = bench.max_over_ranks(torch, dist, world, torch.device("cpu"), ms)
    gbs, sps = bench.job_throughput(world, 4, 2e9, slowest)
    out[rank] = (slowest, gbs, sps)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        slowest, gbs, sps = res[r]
        assert slowest == 150.0
        assert gbs == pytest.approx(2 * 4 * 2e9 / 0.150 / 1e9)
        assert sps == pytest.approx(2 * 4 / 0.150)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(torch, dist, 1, torch.device("cpu"), 12.5) == 12.5
    assert bench.job_throughput(1, 2, 1e9, 1000.0) == pytest.approx((2.0, 2.0))
