"""The replica aggregation of bench.py across ranks (gloo, world size 2, on
CPU): whole-job rate = all ranks' work over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0, 250.0][rank]
    work = [1.0e9, 3.0e9][rank]
    res = (bench.max_over_ranks(ms), bench.sum_over_ranks(work), bench.whole_job_rate(work, ms))
    q.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        mx, sm, rate = out[r]
        assert mx == 250.0 and sm == 4.0e9
        assert abs(rate - 4.0e9 / 0.25) < 1e-3
