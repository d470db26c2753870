"""Multi-GPU runs are replicas: each rank tracks its own streams on its own GPU
with no data-path collective; bench.py only reduces the timed region's length
(max over ranks) and reports units of all ranks / that time.  Exercised here
with world_size 2 on CPU (gloo)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as tmp       # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 150.0][rank]                       # rank 1 is the slow one
    m = bench.max_over_ranks(ms, torch.device("cpu"), world)
    value = bench.job_throughput(64 * 10, world, m)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, m, value))


def test_two_ranks_take_the_slowest_rank_time_and_sum_the_units():
    world = 2
    ctx = tmp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(world))
    for rank, m, value in got:
        assert m == 150.0                           # both ranks see the max
        assert value == pytest.approx(2 * 640 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu"), 1) == 3.5
    assert bench.job_throughput(100, 1, 1000.0) == pytest.approx(100.0)
