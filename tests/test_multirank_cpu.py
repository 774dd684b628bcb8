"""The N > 1 path of bench.py on CPU: two gloo ranks, replicas with no
collective on the data path, barrier and max-over-ranks timing."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, l = bench.dist_setup()
    assert (w, r, l) == (world, rank, rank)
    bench.barrier(w)
    # each rank's "elapsed time"; the job's time is the slowest rank's
    mine = 1.0 + rank
    t = bench.reduce_max(mine, w)
    # replicas: every rank draws its own batched instances (seed offset by rank)
    from paper_2410_06657_gb300 import workloads as W
    first = W.batched(n=2, seed=2410066570 + rank)[0]["params"]
    out[rank] = (t, first["CaE"])
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_replicas():
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0          # max over ranks
    assert res[0][1] != res[1][1]                 # each replica has its own draws
