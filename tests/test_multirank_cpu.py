"""The replicas-only multi-GPU path of bench.py, checked with two gloo ranks on CPU:
the job time is the slowest rank's and the value counts every rank's solves."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = 2.0 if rank == 0 else 3.0            # rank 1 is the slow one
    value, t = bench.whole_job_value(elapsed, steps_per_rank=6, dist=dist)
    q.put((rank, value, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_report_whole_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get() for _ in range(2))
    for rank, value, t in out:
        assert t == 3.0
        assert value == pytest.approx(2 * 6 / 3.0)


def test_single_process_value():
    import bench
    v, t = bench.whole_job_value(4.0, 8, None)
    assert (v, t) == (2.0, 4.0)
