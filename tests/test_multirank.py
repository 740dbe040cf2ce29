"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1) run the whole-job
aggregation the bench uses -- every rank an independent replica, the job's throughput the
units of all ranks over the slowest rank's time -- and its barrier."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_env()[:2] == (rank, world)
    bench.barrier(world)
    value, ms = bench.job_throughput(1000.0, 1.0 + rank, world, device="cpu")  # rank r took 1 + r ms
    out.put((rank, value, ms))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_replicas_aggregate_over_the_slowest_rank():
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
    for rank, value, ms in res:
        assert ms == 2.0  # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 1000.0 / 2e-3)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.job_throughput(500.0, 4.0, 1, device="cpu")
    assert ms == 4.0 and value == pytest.approx(500.0 / 4e-3)
