"""The multi-GPU path of bench.py runs independent replicas (one per rank) and reports the whole
job's throughput against the slowest rank; its rank aggregation is exercised here with two gloo
ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0 + 5.0 * rank, 30.0 - 7.0 * rank]          # rank 1 is slower on the first timing
    mx = bench.max_over_ranks(ms, "cpu")
    value = bench.replica_throughput(1000, 20, mx[0], world)
    out.put((rank, mx, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, value in res:
        assert mx == [15.0, 30.0]
        assert value == pytest.approx(2 * 1000 * 20 / 0.015)
