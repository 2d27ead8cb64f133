"""Multi-rank host logic of bench.py on CPU with the gloo backend
(world size 2): every rank advances its own instance, the job time is the
slowest rank's, and ensemble members are split across ranks without
overlap.  No data-path collective exists; the only collective is the
timing reduction tested here."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 20.0][rank]
    mx = bench.max_over_ranks(dist, local_ms, "cpu")
    mine = bench.shard(48, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out[rank] = (mx, bench.job_throughput(world, 100, mx), gathered, bench.rank_seed(rank))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        mx, thr, gathered, seed = out[r]
        assert mx == 20.0
        assert abs(thr - 2 * 100 / 0.020) < 1e-9
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(48))
        assert not set(gathered[0]) & set(gathered[1])
    assert out[0][3] != out[1][3]


def _ensemble_member(i):
    """Small independent PFC instance i (16^2, seeded, its own dt)."""
    import numpy as np
    rng = np.random.default_rng(100 + i)
    rho = 0.8 + 0.05 * rng.uniform(-1, 1, (16, 16))
    vel = [0.03 * rng.standard_normal((16, 16)) for _ in range(2)]
    return rho, vel, 0.005 * (1 + i)


def _step_member(i):
    from oracle import scheme as S
    rho, vel, dt = _ensemble_member(i)
    P = S.Params(kind=S.PFC, dim=2, h=0.9, s=dt, alpha=0.6, w_damp=0.0)
    r1, v1, info = S.step(rho, vel, P, S.SolverOpts(tol=1e-12, coarsest=4))
    return r1, v1, info["cycles"]


def _shard_worker(rank, world, port, count, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.shard(count, rank, world)
    results = {i: _step_member(i) for i in mine}   # this rank's shard, no data exchange
    gathered = [None] * world
    dist.all_gather_object(gathered, results)
    out[rank] = gathered
    dist.destroy_process_group()


def test_two_gloo_ranks_step_their_shards():
    """The ensemble partition bench.py uses under torchrun, with solver work on
    every rank: two gloo ranks each step their shard of a 5-instance
    ensemble (the oracle stands in for the GPU here); every instance is
    stepped exactly once, by one rank, and the gathered results equal a
    serial stepping of the whole ensemble bit for bit."""
    import numpy as np
    world, count = 2, 5
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, count, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    parts = out[0]
    assert [sorted(p) for p in parts] == [sorted(p) for p in out[1]]
    owners = [i for part in parts for i in part]
    assert sorted(owners) == list(range(count))
    merged = {i: v for part in parts for i, v in part.items()}
    for i in range(count):
        r1, v1, cyc = _step_member(i)
        rg, vg, cg = merged[i]
        assert cg == cyc and np.array_equal(rg, r1) and all(np.array_equal(a, b) for a, b in zip(vg, v1))
