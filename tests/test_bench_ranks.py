"""The multi-process path of the benchmark on CPU: two gloo ranks combine
their step times (maximum) and units (sum) the way the GPU replicas do."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.combine_over_ranks(1.5 + rank, 100.0 * (rank + 1))
    q.put((rank, ms, units))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_combine_time_and_units():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    # every rank sees the slowest time and the work of both
    assert out == [(0, 2.5, 300.0), (1, 2.5, 300.0)]


def test_single_process_returns_its_own_values():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_over_ranks(3.0, 7.0) == (3.0, 7.0)
