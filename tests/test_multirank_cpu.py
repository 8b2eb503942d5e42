"""The N > 1 replica path of bench.py on CPU: two gloo ranks, each timing its
own field, agree on the slowest rank's time and on the whole-job throughput
(weak scaling: world x bytes per rank / the slowest time)."""
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
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_setup() == (world, rank, rank)
        dist.barrier()
        my_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        ms = bench.max_over_ranks(my_ms, world, "cpu")
        value = bench.job_throughput_gbs(1 << 30, 4, ms, world)
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_job_throughput():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    expect_ms = 15.0
    expect_value = world * (1 << 30) * 4 / (expect_ms * 1e-3) / 1e9
    assert dict(out) == {0: (expect_ms, expect_value), 1: (expect_ms, expect_value)}


def test_one_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput_gbs(1000, 2, 1.0, 1) == pytest.approx(2e-3)
