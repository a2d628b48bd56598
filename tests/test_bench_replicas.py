"""bench.py's multi-GPU form on CPU: N independent replicas as gloo ranks (world size 2); the
whole-job rate is all ranks' units over the slowest rank's time, the same on every rank."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [40.0, 50.0][rank]            # the second rank is the slower one
    value, ms_max = bench.replica_rate(tdist, torch.device("cpu"), ms_local, 1000, 4, world)
    tdist.barrier()
    tdist.destroy_process_group()
    q.put((rank, value, ms_max))


def test_replica_rate_takes_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, value, ms_max in res:
        assert ms_max == 50.0
        assert value == pytest.approx(1000 * 2 * 4 / 0.050)


def test_replica_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    value, ms_max = bench.replica_rate(None, None, 25.0, 500, 2, 1)
    assert ms_max == 25.0 and value == pytest.approx(500 * 2 / 0.025)
