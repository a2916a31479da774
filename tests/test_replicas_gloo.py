"""Multi-rank path of bench.py on CPU (gloo, world size 2): replicas take
disjoint patch ids and the job time is the maximum over ranks.  The method
shards by patch with no exchange step, so there is no data-path collective."""
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
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    base = bench.replica_patch_base(rank, 2000)
    ids = torch.arange(base, base + 2000, dtype=torch.int64)
    gathered = [torch.zeros_like(ids) for _ in range(world)]
    dist.all_gather(gathered, ids)
    ms = bench.reduce_max(10.0 + rank, dist, "cpu")
    if rank == 0:
        allids = torch.cat(gathered)
        out.put((int(allids.unique().numel()), int(allids.numel()), ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_disjoint_ids_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    uniq, total, ms = q.get(timeout=10)
    assert uniq == total == 4000
    assert ms == 11.0
