"""The N > 1 bench path on CPU ranks (gloo, world size 2): every rank runs
its own replica; the timed region's duration is the slowest rank's and the
whole-job rate counts every rank's units. No GPU is involved."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    assert bench.dist_env() == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        ms_max = bench.reduce_max(dist, ms, device="cpu")
        rate = bench.whole_job_rate(world, 1000 * 20, ms_max * 1e-3)
        out[rank] = (ms_max, rate)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_sum_the_units():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    ms_max, rate = res[0]
    assert ms_max == 15.0
    assert rate == pytest.approx(2 * 1000 * 20 / 0.015)


def test_single_process_has_no_group():
    import bench

    assert bench.reduce_max(None, 3.5) == 3.5
    assert bench.whole_job_rate(1, 100, 2.0) == 50.0
