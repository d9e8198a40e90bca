"""The multi-GPU form of the benchmark is independent replicas (one handle
per rank, no data-path collective): the host-side logic that combines the
ranks -- the barrier, the maximum of the timed region over ranks and the
whole-job value -- checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp       # noqa: E402


def _free_port() -> int:
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 + 5.0 * rank            # the second rank is the slower one
    dist.barrier()
    ms = bench.max_over_ranks(ms_local, dist, "cpu")
    value = bench.job_value(1000, world, 20, ms)
    out.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_value():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 15.0                                   # the maximum over ranks, on every rank
        assert value == pytest.approx(1000 * 2 * 20 / 15e-3)


def test_single_process_passes_through():
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.job_value(1125000, 1, 500, 1100.0) == pytest.approx(1125000 * 500 / 1.1)

