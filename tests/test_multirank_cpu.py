"""The N > 1 path of bench.py on CPU: two gloo ranks, each solving its own systems, combine only
the slowest time and the total count (weak scaling, no collective on the data path)."""

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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, systems = bench.aggregate_ranks(100.0 + 50.0 * rank, 4 + rank)
    out[rank] = (ms, systems)
    dist.destroy_process_group()


def test_two_ranks_take_max_time_and_sum_systems():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == (150.0, 9) and out[1] == (150.0, 9)


def test_single_process_is_identity():
    import bench
    assert bench.aggregate_ranks(12.5, 4) == (12.5, 4)
