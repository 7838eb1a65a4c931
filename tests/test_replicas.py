"""The multi-GPU path of bench.py is replicas only: every rank solves its own
batch and the ranks share nothing but the barriers and the max-reduction of
the timed region.  This runs that host logic on two gloo ranks on the CPU."""
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


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)     # rank 1 is slower
        value = bench.whole_job_value(12, 10, ms, world)
        out.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 15.0                        # the max over ranks
        assert value == pytest.approx(2 * 12 * 10 / 15e-3)   # whole job, weak scaling


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.whole_job_value(12, 10, 100.0, 1) == pytest.approx(1200.0)
