"""Particle sharding through the CUDA library: two processes share one posterior (each moves half of
the particles; sharded.py drives them with gloo collectives on the host) and must reproduce the
single-context run bit for bit: temperatures, log Z, step size, theta of every particle, the cached
estimates and block sums, and u inside each process's slice. Both processes use the one GPU of the
test box: their kernels never wait on each other (the exchanges are host collectives between
launches), so they only share the device."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STAGES, R = 6, 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    from smc_workloads import small_glm
    return small_glm("logistic", n=20000, p=8, N=1001, m=64, G=4, L=5, x_dtype="bf16", seed=3,
                     theta_scale=0.4)


def _context(wl, **kw):
    import paper_1805_03317_gb300 as S
    from gpu_common import device_arrays
    X, y = device_arrays(wl)
    return S.smc_init(X, y, wl.family, wl.prior_mean, wl.prior_var, N=wl.N, m=wl.m, G=wl.G,
                      L=wl.L, seed=wl.seed, ess_frac=0.5, theta_bar=None, **kw)


def _state(ctx):
    import paper_1805_03317_gb300 as S
    th, u, W = S.smc_get_particles(ctx)
    ell, s2, blk = S.smc_get_cache(ctx)
    st = S.smc_get_status(ctx)
    return dict(theta=th.cpu().numpy(), u=u.cpu().numpy(), W=W.cpu().numpy(),
                ell=ell.cpu().numpy(), sig2=s2.cpu().numpy(), blk=blk.cpu().numpy(),
                status=(st["a"], st["log_z"], st["eps"], st["stage"]))


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        import paper_1805_03317_gb300 as S
        wl = _workload()
        lo, hi = S.shard_bounds(wl.N, world, rank)
        ctx = _context(wl, shard_base=lo, shard_count=hi - lo)
        drv = S.ShardedSMC(ctx, wl.N)
        for _ in range(STAGES):
            drv.stage(R)
        out = _state(ctx)
        out.update(rank=rank, lo=lo, hi=hi, migrated=sum(h["migrated"] for h in drv.history))
        S.smc_free(ctx)
        q.put(out)
    finally:
        dist.destroy_process_group()


def test_two_processes_reproduce_the_single_context_run():
    import paper_1805_03317_gb300 as S
    ctxm = mp.get_context("spawn")
    q = ctxm.Queue()
    port = _free_port()
    procs = [ctxm.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=600) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    wl = _workload()
    ref_ctx = _context(wl)
    for _ in range(STAGES):
        S.smc_reweight(ref_ctx)
        S.smc_resample(ref_ctx)
        S.smc_move(ref_ctx, R)
    ref = _state(ref_ctx)
    S.smc_free(ref_ctx)
    for d in got:
        assert d["status"] == ref["status"]
        for k in ("theta", "W", "ell", "sig2", "blk"):
            assert np.array_equal(d[k], ref[k]), k
        lo, hi = d["lo"], d["hi"]
        assert np.array_equal(d["u"][lo:hi], ref["u"][lo:hi])
    assert sum(d["migrated"] for d in got) > 0
    assert 0.0 < ref["status"][0] <= 1.0
