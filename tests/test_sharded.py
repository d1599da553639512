"""Particle sharding of one posterior over processes (paper_1805_03317_gb300/sharded.py), host
logic on CPU: two or three gloo ranks drive the sharded stage with a host stand-in for the library's
per-process calls (tests/shard_fake.py: the oracle's reweighting, moments and resampling, a toy
move that reads each particle's own u and global index, u kept only inside each slice). The
sharded run must equal the one-process run of the same driver exactly: temperatures, log Z,
ancestors (through the particles they carry), theta, the cached estimates and u."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SHAPE = dict(N=97, p=3, m=6, G=2, n=500, seed=13)  # N odd: uneven slices


def _run(world, rank, group, stages=6):
    import torch.distributed as dist  # noqa: F401
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import shard_fake as F
    from paper_1805_03317_gb300.sharded import ShardedSMC, shard_bounds
    lo, hi = shard_bounds(SHAPE["N"], world, rank)
    ctx = F.FakeCtx(SHAPE["N"], SHAPE["p"], SHAPE["m"], SHAPE["G"], SHAPE["n"], SHAPE["seed"],
                    lo, hi)
    drv = ShardedSMC(ctx, SHAPE["N"], group=group, ops=F)
    for _ in range(stages):
        drv.stage(2)
    return ctx, drv


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ctx, drv = _run(world, rank, None)
        solo = dist.new_group([rank])  # the same driver on one process, for comparison
        ref, rdrv = _run(1, 0, solo)
        out = {
            "rank": rank,
            "same_history": [(h["a"], h["log_z_inc"]) for h in drv.history]
            == [(h["a"], h["log_z_inc"]) for h in rdrv.history],
            "same_theta": np.array_equal(ctx.theta, ref.theta),
            "same_cache": np.array_equal(ctx.ell, ref.ell) and np.array_equal(ctx.sig2, ref.sig2)
            and np.array_equal(ctx.blk, ref.blk),
            "same_u_slice": np.array_equal(ctx.u[ctx.lo:ctx.hi], ref.u[ctx.lo:ctx.hi]),
            "same_status": F_status(ctx) == F_status(ref),
            "migrated": sum(h["migrated"] for h in drv.history),
            "a": ctx.a,
        }
        q.put(out)
    finally:
        dist.destroy_process_group()


def F_status(c):
    return (c.a, c.log_z, c.eps, c.stage)


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reproduce_the_single_process_run(world):
    """world = 3: slices of 32, 32 and 33 particles, rows migrating between every pair of ranks."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = sorted((q.get(timeout=10) for _ in range(world)), key=lambda d: d["rank"])
    for d in got:
        assert d["same_history"] and d["same_status"], d
        assert d["same_theta"] and d["same_cache"] and d["same_u_slice"], d
    assert sum(d["migrated"] for d in got) > 0  # rows really crossed between the ranks
    assert 0.0 < got[0]["a"] <= 1.0


def test_migration_plan_covers_every_remote_ancestor():
    sys.path.insert(0, ROOT)
    from paper_1805_03317_gb300.sharded import migration_plan, owners, shard_bounds
    rng = np.random.default_rng(3)
    N, world = 50, 3
    anc = np.sort(rng.integers(0, N, size=N))
    plan = migration_plan(anc, world)
    own = owners(N, world)
    for r in range(world):
        lo, hi = shard_bounds(N, world, r)
        remote = {j for j in range(lo, hi) if own[anc[j]] != r}
        got = set()
        for s in range(world):
            js, a = plan[s][r]
            assert np.all(own[a] == s) and np.array_equal(a, anc[js]) and np.all(np.diff(js) > 0)
            got |= set(js.tolist())
        assert got == remote
    assert [shard_bounds(10, 3, r) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
