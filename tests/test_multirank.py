"""Host-side logic of the multi-GPU bench path on CPU: world size 2 over gloo.

Each rank advances its own cavity (replicas; the method has no exchange between
independent cavities).  The job time is the max over ranks and the throughput is the
sum of the node updates of all ranks divided by it.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    bench.barrier(dist)
    elapsed = 1.0 + rank  # rank 1 is the slow one
    lups = 1000.0 * (rank + 1)
    t = bench.max_over_ranks(dist, elapsed)
    total = bench.sum_over_ranks(dist, lups)
    out[rank] = (w, r, t, total)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_aggregation_over_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(90)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        w, rank, t, total = res[r]
        assert (w, rank) == (world, r)
        assert t == 2.0          # the slowest rank sets the job time
        assert total == 3000.0   # every rank's node updates count


def test_single_process_defaults():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    w, r, local = bench.dist_env()
    assert (w, r) == (1, 0)
    assert bench.init_dist(w, "gloo") is None
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.sum_over_ranks(None, 7.0) == 7.0
