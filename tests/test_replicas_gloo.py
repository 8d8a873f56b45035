"""Multi-process aggregation of the benchmark's replicas, on CPU with gloo
(world size 2): the job time is the slowest rank's, rays add up."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2504_21627_gb300 import replicas
    ms, rays, value = replicas.aggregate(10.0 * (rank + 1), 1000 * (rank + 1))
    dist.barrier()
    q.put((rank, ms, rays, value, replicas.shard(10, rank, world)))
    dist.destroy_process_group()


def test_aggregate_over_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=60) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rays, value, sh in res:
        assert ms == 20.0 and rays == 3000
        assert abs(value - 3000 / 0.020 / 1e6) < 1e-12
    assert res[0][4] == (0, 5) and res[1][4] == (5, 10)


def test_single_process_fallback():
    from paper_2504_21627_gb300 import replicas
    assert replicas.aggregate(4.0, 4_000_000) == (4.0, 4_000_000, 1000.0)
    assert replicas.shard(7, 2, 3) == (5, 7)
