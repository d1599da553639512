"""A host-only stand-in for the CUDA library's per-process calls, for CPU tests of the sharded
driver (paper_1805_03317_gb300/sharded.py) on gloo ranks.

The stage arithmetic that every process repeats on the full arrays is the oracle's (temperature
search and reweighting, weighted moments, systematic resampling with the Philox uniform of the
stage). The moves are a deterministic toy that depends on each particle's own u and its global
index, so that a wrong migration of u, a wrong slice or a wrong index changes the result. u is
kept current only inside the process's slice: every other row holds -1, as on a real process
whose copy of those rows is stale."""
from __future__ import annotations

import math

import numpy as np
import torch

from oracle import oracle as O


class FakeCtx:
    def __init__(self, N, p, m, G, n, seed, lo, hi, a_tau=0.5):
        rng = np.random.default_rng(seed)
        self.N, self.p, self.m, self.G, self.n, self.seed = N, p, m, G, n, seed
        self.lo, self.hi, self.tau = lo, hi, a_tau
        self.device = "cpu"
        self.theta = rng.standard_normal((N, p))
        self.u = rng.integers(0, n, size=(N, m)).astype(np.int32)
        self.u_prev = self.u.copy()
        self.logW = np.full(N, -math.log(N))
        self.W = np.full(N, 1.0 / N)
        self.a, self.log_z, self.eps, self.stage = 0.0, 0.0, 0.3, 0
        self.acc = [0, 0]
        # like the library, every process starts from all N particles and their estimates;
        # afterwards it keeps u current only inside its slice
        self._refresh(range(N))
        self._poison()

    def _poison(self):
        keep = self.u[self.lo:self.hi].copy()
        self.u[:] = -1
        self.u[self.lo:self.hi] = keep

    def _estimates(self, i):
        """Toy cached estimates of particle i (depend on theta_i and its u row)."""
        th, ui = self.theta[i], self.u[i].astype(np.int64)
        s = float(th @ th)
        ell = -0.5 * s * self.n / 50.0 + 0.01 * float(ui.sum() % 13)
        sig2 = 0.05 * s + 1e-3 * float(ui.sum() % 7)
        blk = np.empty((self.G, 2))
        blk[:, 0] = ell / self.G
        blk[:, 1] = sig2 / self.G
        return ell, sig2, blk

    def _refresh(self, idx):
        if not hasattr(self, "ell"):
            self.ell = np.zeros(self.N)
            self.sig2 = np.zeros(self.N)
            self.blk = np.zeros((self.N, self.G, 2))
        for i in idx:
            if self.u[i, 0] < 0:  # a stale row: this process never computes with it
                continue
            self.ell[i], self.sig2[i], self.blk[i] = self._estimates(i)


def _h(*v):
    """A 64-bit mix of integers (splitmix64 steps)."""
    x = 0x9E3779B97F4A7C15
    for t in v:
        x = (x ^ (int(t) & 0xFFFFFFFFFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF
        x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        x = z ^ (z >> 31)
    return x


# -- the calls the sharded driver makes (same names as the CUDA binding) -------------------------
def smc_reweight(c: FakeCtx):
    c.stage += 1
    a_new, logW, W, lz, ess = O.reweight(c.logW, c.ell, c.sig2, c.a, c.tau)
    c.a, c.logW, c.W = a_new, logW, W
    c.log_z += lz
    return a_new, lz, ess


def smc_resample(c: FakeCtx, anc: torch.Tensor):
    U = O.uniform(O.r64(c.seed, O.TAG_RESAMPLE, O.stage_move(c.stage, 0), 0, 0))
    a = O.resample(c.W, U).astype(np.int64)
    c.u_prev = c.u.copy()
    c.theta, c.u = c.theta[a].copy(), c.u[a].copy()
    c.ell, c.sig2, c.blk = c.ell[a].copy(), c.sig2[a].copy(), c.blk[a].copy()
    c.logW = np.full(c.N, -math.log(c.N))
    c.W = np.full(c.N, 1.0 / c.N)
    anc.copy_(torch.from_numpy(a.astype(np.int32)))


def smc_shard_gather_u(c: FakeCtx, idx: torch.Tensor, before_resample: bool):
    src = c.u_prev if before_resample else c.u
    return torch.from_numpy(src[idx.numpy().astype(np.int64)].copy())


def smc_shard_scatter_u(c: FakeCtx, idx: torch.Tensor, rows: torch.Tensor):
    c.u[idx.numpy().astype(np.int64)] = rows.numpy()


def smc_move(c: FakeCtx, R: int):
    c.acc = [0, 0]
    c._poison()  # rows outside the slice are stale after resampling
    for r in range(R):
        for i in range(c.lo, c.hi):
            assert c.u[i, 0] >= 0, "a row of this slice was not migrated"
            h = _h(c.seed, c.stage, r, i)
            c.u[i, h % c.m] = (h >> 8) % c.n
            c.acc[0] += (h >> 40) & 1
            if (h >> 41) & 1:
                k = int(c.u[i].astype(np.int64).sum() % 97)
                c.theta[i] += c.eps * 0.1 * np.cos(k + i + np.arange(c.p))
                c.acc[1] += 1
        c._refresh(range(c.lo, c.hi))
    return c.acc[0] / ((c.hi - c.lo) * R), c.acc[1] / ((c.hi - c.lo) * R)


def smc_move_accepts(c: FakeCtx):
    return c.acc[0], c.acc[1]


def smc_finish_moves(c: FakeCtx, R: int, acc_u: int, acc_theta: int):
    c.eps *= min(2.0, max(0.5, math.exp(acc_theta / (c.N * R) - 0.65)))


def smc_shard_export(c: FakeCtx, count: int):
    s = slice(c.lo, c.hi)
    return (torch.from_numpy(c.theta[s].copy()), torch.from_numpy(c.ell[s].copy()),
            torch.from_numpy(c.sig2[s].copy()), torch.from_numpy(c.blk[s].copy()))


def smc_shard_import(c: FakeCtx, theta, ell, sigma2, blocks):
    c.theta = theta.numpy().copy()
    c.ell = ell.numpy().copy()
    c.sig2 = sigma2.numpy().copy()
    c.blk = blocks.numpy().copy()


def smc_get_status(c: FakeCtx):
    return {"a": c.a, "log_z": c.log_z, "stage": c.stage, "eps": c.eps}
