"""The N > 1 timing rule of the benchmark (replicas, max over ranks, units of
all ranks) on two gloo ranks on the CPU."""
import os

import pytest
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1311_3004_gb300.replicas import job_throughput
    secs = [2.0, 3.0][rank]
    units = [100.0, 50.0][rank]
    q.put((rank, job_throughput(secs, units)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_job_throughput():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        value, t, world = out[r]
        assert world == 2 and t == 3.0 and value == pytest.approx(150.0 / 3.0)


def test_single_process_fallback():
    from paper_1311_3004_gb300.replicas import job_throughput
    assert job_throughput(2.0, 10.0) == (5.0, 2.0, 1)
