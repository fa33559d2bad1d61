"""The N > 1 benchmark path on the CPU: two gloo ranks, each with its own material
(no data exchange), the slowest rank's time as the job time, and the job throughput
counting every rank's blocks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, queue):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms = 10.0 + 5.0 * r                       # rank 1 is slower
    job_ms = bench.max_over_ranks(ms, w)
    queue.put((r, w, bench.rank_material_seed(r), job_ms, bench.job_throughput(1_000_000, w, job_ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_and_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    seeds = {o[2] for o in out}
    assert len(seeds) == world                                  # each rank its own material
    assert all(o[3] == pytest.approx(15.0) for o in out)        # slowest rank's time
    assert all(o[4] == pytest.approx(2 * 1_000_000 / 15e-3 / 1e6) for o in out)

