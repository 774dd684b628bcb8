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


def _replica(rank, world, port, out):
    """One rank advancing its own replica (the FP64 oracle stands in for the
    GPU library on a CPU-only host), timed as the bench times a step."""
    import time
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2410_06657_gb300 import workloads as W
    w, r, _ = bench.dist_setup()
    p = dict(W.batched(n=1, seed=2410066570 + r)[0]["params"], nx=32, ny=16, R0=5.0, precision=W.FP64)
    o = oracle.Oracle(p)
    o.init_droplet(5.0, *W.sessile_center(32, 5.0, p["theta_deg"]), 0)
    steps = 20
    bench.barrier(w)
    t0 = time.perf_counter()
    o.step(steps)
    el = bench.reduce_max(time.perf_counter() - t0, w)
    value = w * p["nx"] * p["ny"] * steps / el / 1e6      # the bench's whole-job MLUPS
    out[rank] = (value, o.observables()["mass"], p["CaE"])
    dist.destroy_process_group()


def test_two_gloo_ranks_advance_their_own_replicas():
    """Each rank steps its own instance (its own parameter draws), the job's
    rate counts every rank's lattice updates over the slowest rank's time,
    and a rank's result is that of its instance run alone."""
    import oracle
    from paper_2410_06657_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_replica, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] > 0.0           # one whole-job rate, agreed by both ranks
    assert res[0][2] != res[1][2]                 # distinct replicas
    for r in range(world):
        p = dict(W.batched(n=1, seed=2410066570 + r)[0]["params"], nx=32, ny=16, R0=5.0, precision=W.FP64)
        o = oracle.Oracle(p)
        o.init_droplet(5.0, *W.sessile_center(32, 5.0, p["theta_deg"]), 0)
        o.step(20)
        assert o.observables()["mass"] == res[r][1]
