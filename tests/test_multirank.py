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
