"""The N > 1 benchmark path runs independent replicas (no data-path
collective): only the timing is reduced.  Checked with two gloo ranks on CPU:
every rank gets the max step time and value = N * cells / max time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, kms, value = bench.replica_aggregate(1.0 + rank, 0.5 + rank, 1000, world, torch.device("cpu"))
    q.put((rank, ms, kms, value))
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, kms, value in res:
        assert ms == 2.0 and kms == 1.5
        assert value == pytest.approx(2 * 1000 / 2e-3)
