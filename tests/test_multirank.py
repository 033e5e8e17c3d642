"""The multi-GPU path on CPU: world size 2 with the gloo backend.  Streams are sharded
over ranks with no exchange on the data path (weak scaling); the only collectives are
the benchmark's barrier and the max of the per-rank times.  Checks that the shards are
disjoint and cover the workload, and that bench.py's reduced time is the slowest rank's
and its whole-job value counts every rank's doubles."""
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
    import bench
    from paper_2106_02504_gb300 import workloads as W
    seeds = torch.from_numpy(W.rank_seeds(rank, world, n).view(np.int64))
    gathered = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    dist.barrier()
    # bench.py's reduction and whole-job value, as every rank runs them
    ms = bench.max_over_ranks(10.0 + rank, dist, torch.device("cpu"))   # per-rank step time
    value = bench.whole_job_doubles_per_s(n, world, ms)
    if rank == 0:
        out.put((torch.cat(gathered).numpy().view(np.uint64).tolist(), ms, value))
    dist.destroy_process_group()


def test_two_rank_sharding_with_gloo():
    world, n = 2, 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    seeds, tmax, value = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(seeds) == list(range(1, world * n + 1))   # disjoint and complete
    assert tmax == 11.0                                      # the slowest rank sets the time
    # all ranks' doubles (5120 per stream and step) over the slowest rank's time
    assert value == world * n * 5120 / 11e-3


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.max_over_ranks(7.5, None, None) == 7.5
    assert bench.whole_job_doubles_per_s(1 << 20, 1, 7.85) == (1 << 20) * 5120 / 7.85e-3


def test_rank_seeds_bounds():
    from paper_2106_02504_gb300 import workloads as W
    assert W.rank_seeds(0, 1, 3).tolist() == [1, 2, 3]
    assert W.rank_seeds(1, 2, 3).tolist() == [4, 5, 6]
    with pytest.raises(ValueError):
        W.rank_seeds(2, 2, 3)
