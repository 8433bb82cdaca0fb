"""The multi-rank (N > 1) path on CPU: two gloo ranks, each a replica with
its own timed region and unit count; the job throughput is the sum of the
units over the slowest rank's time, and only rank 0 reports."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2407_18015_gb300 import replicas
    r, w = replicas.init("gloo")
    assert (r, w) == (rank, world)
    replicas.barrier()
    ms = 10.0 + 5.0 * rank          # rank 1 is the slowest
    units = 1000 * (rank + 1)
    max_ms, total, value = replicas.job_throughput(ms, units)
    out.put((rank, max_ms, total, value))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, max_ms, total, value in res:
        assert max_ms == 15.0 and total == 3000.0
        assert value == pytest.approx(3000.0 / 0.015)


def test_single_process_is_identity():
    from paper_2407_18015_gb300 import replicas
    max_ms, total, value = replicas.job_throughput(4.0, 10)
    assert (max_ms, total) == (4.0, 10.0) and value == pytest.approx(2500.0)
