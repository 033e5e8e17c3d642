"""The multi-GPU path on CPU: world size 2 with the gloo backend.  Streams are sharded
over ranks with no exchange on the data path (weak scaling); the only collectives are
the benchmark's barrier and the max of the per-rank times.  Checks that the shards are
disjoint and cover the workload, and that the reduced time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2106_02504_gb300 import workloads as W
    seeds = torch.from_numpy(W.rank_seeds(rank, world, n).view(np.int64))
    gathered = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    t = torch.tensor([10.0 + rank])          # per-rank step time
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((torch.cat(gathered).numpy().view(np.uint64).tolist(), float(t.item())))
    dist.destroy_process_group()


def test_two_rank_sharding_with_gloo():
    world, n = 2, 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    seeds, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(seeds) == list(range(1, world * n + 1))   # disjoint and complete
    assert tmax == 11.0                                      # the slowest rank sets the time


def test_rank_seeds_bounds():
    from paper_2106_02504_gb300 import workloads as W
    assert W.rank_seeds(0, 1, 3).tolist() == [1, 2, 3]
    assert W.rank_seeds(1, 2, 3).tolist() == [4, 5, 6]
    with pytest.raises(ValueError):
        W.rank_seeds(2, 2, 3)
