"""The replica path of bench.py on CPU: two gloo ranks, each with its own time; the whole-job
rate is the units of all ranks over the slowest rank's time, the same on every rank."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [2.0, 5.0][rank]
    rate, slowest = bench.job_rate(10, seconds, dist, torch.device("cpu"))
    q.put((rank, rate, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_takes_max_over_two_gloo_ranks():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, slowest in got:
        assert slowest == 5.0
        assert rate == pytest.approx(2 * 10 / 5.0)


def test_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(7, 2.0) == (3.5, 2.0)
