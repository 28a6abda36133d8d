"""The multi-rank benchmark path on CPU with the gloo backend, world size 2: every
rank steps its own shard (a batch drawn from its own seed, no data-path collective);
the timed region is the maximum over ranks and the whole-job rate counts all ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, _ = bench.make_workload("small", rank)
    t_ms = 100.0 + 50.0 * rank                      # per-rank timed region
    tmax = bench.max_over_ranks(t_ms, world)
    rate = bench.whole_job_rate(b.rbc_equivalents(), world, 4, tmax)
    out[rank] = (tmax, rate, float(b.x[0, 0]), b.ncells)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_aggregate():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    (t0, r0, x0, n0), (t1, r1, x1, n1) = out[0], out[1]
    assert t0 == t1 == 150.0                          # max over ranks
    assert n0 == n1 == 64 and x0 != x1                # equal shard sizes, different seeds
    assert r0 == r1 == pytest.approx(64 * 2 * 4 / 0.150)
