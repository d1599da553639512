"""One posterior's particles split over several processes (one GPU each): Algorithm 2 with the
moves of each stage (Algorithm 1, the expensive part) divided between the processes.

Every process holds a context with all N particles, created with the same problem and seed and
its own slice [lo, hi) (smc_config.shard_base / shard_count). A stage then runs as

    reweight (temperature search, weights, log Z, mass matrix)  every process, on the full arrays
    resample                                                    every process: identical ancestors
    migrate u                 the u rows of ancestors that lived on another process, point to point
    move                                                        each process its own slice only
    accept counts             all-reduce (sum), then the step-size update on every process
    gather                    all-gather of the slices' theta, l_hat, sigma2_hat and block sums

The reweighting and resampling see identical inputs on every process, so the temperatures,
weights and integer ancestors agree exactly; the moves use the particles' global indices in the
counter-based random streams, so a sharded run reproduces the single-process run bit for bit. The
exchanged volumes per stage are 16N + 16NG + 4Np bytes in the all-gather (FP64 estimates, block
sums, FP32 theta) and 4m bytes per migrated particle.

The collectives are torch.distributed's (NCCL between GPUs: device tensors; gloo: host tensors).
`ops` supplies the per-process calls (default: the CUDA library's binding, smc.py)."""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from . import smc as _smc


def shard_bounds(N: int, world: int, rank: int) -> tuple[int, int]:
    """Slice [lo, hi) of rank `rank` when N particles are split over `world` processes."""
    return (rank * N) // world, ((rank + 1) * N) // world


def owners(N: int, world: int) -> np.ndarray:
    """owner[i] = the rank whose slice holds particle i."""
    own = np.empty(N, dtype=np.int64)
    for r in range(world):
        lo, hi = shard_bounds(N, world, r)
        own[lo:hi] = r
    return own


def migration_plan(anc: np.ndarray, world: int):
    """From the replicated ancestors anc [N] (new particle j descends from anc[j]): for every pair
    (source s, destination r != s) the new particles j of r's slice whose ancestor lives in s's
    slice, in increasing j, and their ancestors. Returns plan[s][r] = (j array, anc[j] array)."""
    N = anc.shape[0]
    own = owners(N, world)
    src = own[anc]
    plan = [[(np.empty(0, np.int64), np.empty(0, np.int64)) for _ in range(world)]
            for _ in range(world)]
    for r in range(world):
        lo, hi = shard_bounds(N, world, r)
        js = np.arange(lo, hi)
        for s in range(world):
            if s == r:
                continue
            sel = js[src[lo:hi] == s]
            plan[s][r] = (sel, anc[sel])
    return plan


class ShardedSMC:
    """Drives one process's context in a sharded run. ctx: this process's context (created with
    shard_base = lo, shard_count = hi - lo from shard_bounds); N: the total particle count.
    group: a torch.distributed process group (None: the default group, or one process when
    torch.distributed is not initialised)."""

    def __init__(self, ctx, N: int, group=None, ops=None):
        self.ctx = ctx
        self.N = N
        self.ops = ops if ops is not None else _smc
        self.group = group
        self.dist = dist.is_available() and dist.is_initialized()
        self.world = dist.get_world_size(group) if self.dist else 1
        self.rank = dist.get_rank(group) if self.dist else 0
        self.lo, self.hi = shard_bounds(N, self.world, self.rank)
        backend = dist.get_backend(group) if self.dist else "none"
        self.on_device = backend == "nccl"
        self.history = []

    # -- collectives ------------------------------------------------------------------------------
    def _comm(self, t: torch.Tensor) -> torch.Tensor:
        return t if self.on_device else t.cpu()

    def _all_reduce_sum(self, values) -> list[int]:
        t = self._comm(torch.tensor(values, dtype=torch.int64,
                                    device=getattr(self.ctx, "device", "cpu")))
        if self.world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return [int(v) for v in t.tolist()]

    def _all_gather_slices(self, local: torch.Tensor) -> torch.Tensor:
        """The full [N, ...] array from every process's slice (slices padded to a common length)."""
        if self.world == 1:
            return local
        width = (self.N + self.world - 1) // self.world
        pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype,
                          device=local.device)
        pad[: local.shape[0]] = local
        pad = self._comm(pad)
        parts = [torch.empty_like(pad) for _ in range(self.world)]
        dist.all_gather(parts, pad, group=self.group)
        out = [parts[r][: shard_bounds(self.N, self.world, r)[1] - shard_bounds(self.N, self.world, r)[0]]
               for r in range(self.world)]
        return torch.cat(out).to(local.device)

    # -- the stage --------------------------------------------------------------------------------
    def _migrate(self, anc: torch.Tensor) -> int:
        """Send the u rows of this process's old particles that are now ancestors of another
        process's new particles, and receive the rows of its own new particles whose ancestors
        lived elsewhere. Returns the number of rows received."""
        if self.world == 1:
            return 0
        plan = migration_plan(anc.cpu().numpy().astype(np.int64), self.world)
        me, m = self.rank, self.ctx.m
        send_idx = np.concatenate([plan[me][r][1] for r in range(self.world)])
        send_counts = [len(plan[me][r][0]) * m for r in range(self.world)]
        recv_counts = [len(plan[s][me][0]) * m for s in range(self.world)]
        dev = getattr(self.ctx, "device", "cpu")
        if send_idx.size:
            rows = self.ops.smc_shard_gather_u(self.ctx, torch.from_numpy(send_idx), True)
        else:
            rows = torch.empty(0, m, dtype=torch.int32, device=dev)
        send = self._comm(rows.reshape(-1).contiguous())
        recv = torch.empty(sum(recv_counts), dtype=torch.int32, device=send.device)
        dist.all_to_all_single(recv, send, recv_counts, send_counts, group=self.group)
        recv_j = np.concatenate([plan[s][me][0] for s in range(self.world)])
        if recv_j.size:
            self.ops.smc_shard_scatter_u(self.ctx, torch.from_numpy(recv_j),
                                         recv.reshape(-1, m).to(dev))
        return int(recv_j.size)

    def stage(self, R: int) -> dict:
        """One stage of Algorithm 2 over all processes' particles; returns the temperature, the
        log-evidence increment, the ESS, the global acceptance rates and the rows migrated."""
        ops, ctx = self.ops, self.ctx
        a, lz, ess = ops.smc_reweight(ctx)
        anc = torch.empty(self.N, dtype=torch.int32, device=getattr(ctx, "device", "cpu"))
        ops.smc_resample(ctx, anc)
        migrated = self._migrate(anc)
        ops.smc_move(ctx, R)
        acc_u, acc_t = self._all_reduce_sum(list(ops.smc_move_accepts(ctx)))
        ops.smc_finish_moves(ctx, R, acc_u, acc_t)
        th, ell, s2, blk = ops.smc_shard_export(ctx, self.hi - self.lo)
        ops.smc_shard_import(ctx, self._all_gather_slices(th), self._all_gather_slices(ell),
                             self._all_gather_slices(s2), self._all_gather_slices(blk))
        rec = {"a": a, "log_z_inc": lz, "ess": ess, "acc_u": acc_u / (self.N * R),
               "acc_theta": acc_t / (self.N * R), "migrated": migrated}
        self.history.append(rec)
        return rec

    def run(self, R: int, max_stages: int = 1000) -> dict:
        """Stages until the temperature reaches 1; returns the context's status."""
        while self.ops.smc_get_status(self.ctx)["a"] < 1.0 and len(self.history) < max_stages:
            self.stage(R)
        return self.ops.smc_get_status(self.ctx)
