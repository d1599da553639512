"""Python binding of the C ABI (include/subsmc.h): same entry-point names, argument marshalling only.

Device buffers are torch CUDA tensors; the library computes everything in its own kernels. The
functions ``smc_init`` ... ``smc_launch_count`` mirror the C entry points one for one;
``SubsampledSMC`` bundles them around one context for convenience.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import DTYPE, FAMILY, SmcConfig, SmcProblem, check

_TORCH_X = {torch.float64: "f64", torch.float32: "f32", torch.bfloat16: "bf16"}
RESAMPLING = {"systematic": 0, "multinomial": 1}
THETA_MOVE = {"hmc": 0, "rw": 1}


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream_handle(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """Owns one smc_ctx; the handle is passed to the module-level entry points."""

    def __init__(self, handle: ctypes.c_void_p, N: int, m: int, G: int, p: int, n: int,
                 state_dtype: torch.dtype, device: torch.device, keepalive, owned: bool = True):
        self.handle = handle
        self.N, self.m, self.G, self.p, self.n = N, m, G, p, n
        self.state_dtype = state_dtype
        self.device = device
        self._keepalive = keepalive
        self.owned = owned  # False: a problem of a Batch, freed with the batch

    def __del__(self):
        try:
            if self.owned:
                smc_free(self)
        except Exception:
            pass


# ------------------------------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ------------------------------------------------------------------------------------------------
def smc_init(X: torch.Tensor, y: torch.Tensor, family: str, prior_mean, prior_var, *, N: int,
             m: int, G: int, L: int, seed: int, ess_frac: float = 0.5, noise_sigma: float = 1.0,
             dof: float = 5.0,
             theta_bar=None, search_k: int = 16, search_rounds: int = 10, eps0: float = 0.0,
             tile_hint: int = 0, hmc_kernel: int = 0, cv_kernel: int = 0,
             cv_order: int = 2, cv_centre: int = 0, full_data: bool = False,
             resampling: str = "systematic", grid_points: int = 0, grid_decades: float = 0.0,
             theta_move: str = "hmc", eps_jitter: float = 0.0, shard_base: int = 0,
             shard_count: int = 0, stream=None) -> Context:
    """Create a context (Algorithm 2 step 1) on X's device; the fields mirror smc_problem and
    smc_config in include/subsmc.h.

    X: [n, p] CUDA tensor (float64, float32 or bfloat16 storage), y: [n]. family: "logistic",
    "probit", "poisson", "gaussian" (known sd noise_sigma) or "student_t" (dof, scale
    noise_sigma). N particles, subsample size m, G blocks of u, L leapfrog steps, seed of the
    counter-based random streams, ESS target ess_frac * N. theta_bar: control-variate centre
    (None: the posterior mode by Newton's method on the device). Options of the paper: cv_order
    (2 or 1), cv_centre (0 fixed, 1 re-centred after each reweighting as in Algorithm 2, 2 before
    it), resampling ("systematic" or "multinomial"), grid_points / grid_decades (the grid
    temperature rule), theta_move ("hmc" or "rw"), eps_jitter (0: 0.3; negative: fixed step),
    full_data (the full-data comparison method). Tuning: search_k, search_rounds, eps0, tile_hint,
    hmc_kernel, cv_kernel (0 = automatic). shard_base / shard_count: this process moves only
    particles [shard_base, shard_base + shard_count) of the N (sharded.py drives such contexts)."""
    lib = _abi.load()
    if not X.is_cuda or X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a 2-D CUDA tensor with unit column stride")
    x_dtype = _TORCH_X[X.dtype]
    y_dtype = torch.float64 if x_dtype == "f64" else torch.float32
    y = y.to(device=X.device, dtype=y_dtype).contiguous()
    n, p = X.shape
    pm = np.ascontiguousarray(prior_mean, dtype=np.float64)
    pv = np.ascontiguousarray(prior_var, dtype=np.float64)
    prob = SmcProblem(FAMILY[family], n, p, X.data_ptr(), DTYPE[x_dtype], X.stride(0),
                      y.data_ptr(), _dp(pm), _dp(pv), float(noise_sigma), float(dof))
    cfg = SmcConfig(N, m, G, L, float(ess_frac), int(seed) & ((1 << 64) - 1), search_k,
                    search_rounds, float(eps0), tile_hint, hmc_kernel, cv_kernel,
                    int(cv_order), int(cv_centre), 1 if full_data else 0,
                    RESAMPLING[resampling], int(grid_points), float(grid_decades),
                    THETA_MOVE[theta_move], float(eps_jitter), int(shard_base), int(shard_count))
    tb = None
    tb_ptr = None
    if theta_bar is not None:
        tb = np.ascontiguousarray(theta_bar, dtype=np.float64)
        tb_ptr = _dp(tb)
    handle = ctypes.c_void_p()
    with torch.cuda.device(X.device):
        rc = lib.smc_init(ctypes.byref(handle), ctypes.byref(prob), ctypes.byref(cfg), tb_ptr,
                          _stream_handle(stream))
    check(rc, "smc_init", None)
    state = torch.float64 if x_dtype == "f64" else torch.float32
    return Context(handle, N, m, G, p, n, state, X.device, (y, pm, pv))


def smc_free(ctx: Context) -> None:
    if ctx.handle and ctx.owned:
        _abi.load().smc_free(ctx.handle)
        ctx.handle = ctypes.c_void_p()


def smc_reweight(ctx: Context):
    a, lz, ess = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(_abi.load().smc_reweight(ctx.handle, ctypes.byref(a), ctypes.byref(lz),
                                   ctypes.byref(ess)), "smc_reweight", ctx.handle)
    return a.value, lz.value, ess.value


def smc_resample(ctx: Context, ancestors: torch.Tensor | None = None) -> None:
    check(_abi.load().smc_resample(ctx.handle, _ptr(ancestors)), "smc_resample", ctx.handle)


def smc_move(ctx: Context, R: int):
    au, at = ctypes.c_double(), ctypes.c_double()
    check(_abi.load().smc_move(ctx.handle, R, ctypes.byref(au), ctypes.byref(at)), "smc_move",
          ctx.handle)
    return au.value, at.value


def smc_move_adaptive(ctx: Context, R_max: int, rho_max: float = 0.1, quantile: float = 0.9):
    """Moves until the quantile of the componentwise start-to-current correlations is at most
    rho_max (or R_max moves); returns (moves made, u acceptance, theta acceptance)."""
    r, au, at = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
    check(_abi.load().smc_move_adaptive(ctx.handle, int(R_max), float(rho_max), float(quantile),
                                        ctypes.byref(r), ctypes.byref(au), ctypes.byref(at)),
          "smc_move_adaptive", ctx.handle)
    return r.value, au.value, at.value


def smc_stage(ctx: Context, R: int, use_graph: bool = True):
    """One stage (reweight, resample, R moves) without host synchronisation; with use_graph the
    stage is replayed as one CUDA graph after its first capture."""
    check(_abi.load().smc_stage(ctx.handle, int(R), 1 if use_graph else 0), "smc_stage",
          ctx.handle)


def loglik_est(ctx: Context, theta: torch.Tensor, u: torch.Tensor):
    B = theta.shape[0]
    theta = theta.to(ctx.state_dtype).contiguous()
    u = u.to(torch.int32).contiguous()
    ell = torch.empty(B, dtype=torch.float64, device=theta.device)
    s2 = torch.empty_like(ell)
    check(_abi.load().loglik_est(ctx.handle, B, _ptr(theta), _ptr(u), _ptr(ell), _ptr(s2)),
          "loglik_est", ctx.handle)
    return ell, s2


def loglik_grad(ctx: Context, theta: torch.Tensor, u: torch.Tensor, a: float):
    B = theta.shape[0]
    theta = theta.to(ctx.state_dtype).contiguous()
    u = u.to(torch.int32).contiguous()
    grad = torch.empty_like(theta)
    ell = torch.empty(B, dtype=torch.float64, device=theta.device)
    s2 = torch.empty_like(ell)
    check(_abi.load().loglik_grad(ctx.handle, B, _ptr(theta), _ptr(u), float(a), _ptr(grad),
                                  _ptr(ell), _ptr(s2)), "loglik_grad", ctx.handle)
    return grad, ell, s2


def loglik_full(ctx: Context, theta: torch.Tensor, a: float = 1.0):
    """Full-data l(theta) [B] float64 and the gradient of a l + log p [B, p] float32 (tensor
    cores; BF16 storage, p <= 64)."""
    B = theta.shape[0]
    theta = theta.to(torch.float32).contiguous()
    ell = torch.empty(B, dtype=torch.float64, device=theta.device)
    grad = torch.empty_like(theta)
    check(_abi.load().loglik_full(ctx.handle, B, _ptr(theta), float(a), _ptr(ell), _ptr(grad)),
          "loglik_full", ctx.handle)
    return grad, ell


def loglik_fwd(ctx: Context, theta: torch.Tensor, u: torch.Tensor):
    """l_hat, sigma2_hat [B] float64 and the per-row d, r [B, m] (state type) kept for loglik_bwd."""
    B = theta.shape[0]
    theta = theta.to(ctx.state_dtype).contiguous()
    u = u.to(torch.int32).contiguous()
    ell = torch.empty(B, dtype=torch.float64, device=theta.device)
    s2 = torch.empty_like(ell)
    d = torch.empty(B, ctx.m, dtype=ctx.state_dtype, device=theta.device)
    r = torch.empty_like(d)
    check(_abi.load().loglik_fwd(ctx.handle, B, _ptr(theta), _ptr(u), _ptr(ell), _ptr(s2), _ptr(d),
                                 _ptr(r)), "loglik_fwd", ctx.handle)
    return ell, s2, d, r


def loglik_bwd(ctx: Context, theta: torch.Tensor, u: torch.Tensor, d: torch.Tensor,
               r: torch.Tensor, g_ell: torch.Tensor, g_sig2: torch.Tensor):
    """Gradient [B, p] (state type) of g_ell . l_hat + g_sig2 . sigma2_hat from saved d, r."""
    theta = theta.to(ctx.state_dtype).contiguous()
    u = u.to(torch.int32).contiguous()
    d = d.contiguous()
    r = r.contiguous()
    ge = g_ell.to(device=theta.device, dtype=torch.float64).contiguous()
    gs = g_sig2.to(device=theta.device, dtype=torch.float64).contiguous()
    grad = torch.empty_like(theta)
    check(_abi.load().loglik_bwd(ctx.handle, theta.shape[0], _ptr(theta), _ptr(u), _ptr(d),
                                 _ptr(r), _ptr(ge), _ptr(gs), _ptr(grad)), "loglik_bwd", ctx.handle)
    return grad


class SubsampledLoglik(torch.autograd.Function):
    """(l_hat, sigma2_hat) of the difference estimator as a differentiable function of theta for a
    fixed subsample u (Sec. 3.2). The forward kernel saves each row's increment d_j and its
    derivative r_j; the backward kernel gathers the particle's rows again by u and forms the exact
    gradient from them (no tape through the estimator, no finite differences).
    Usage: ell, s2 = SubsampledLoglik.apply(theta, u, ctx)."""

    @staticmethod
    def forward(fctx, theta, u, ctx):
        ell, s2, d, r = loglik_fwd(ctx, theta.detach(), u)
        fctx.save_for_backward(theta.detach(), u, d, r)
        fctx.smc_ctx = ctx
        fctx.in_dtype = theta.dtype
        return ell, s2

    @staticmethod
    def backward(fctx, g_ell, g_sig2):
        theta, u, d, r = fctx.saved_tensors
        B = theta.shape[0]
        if g_ell is None:
            g_ell = torch.zeros(B, dtype=torch.float64, device=theta.device)
        if g_sig2 is None:
            g_sig2 = torch.zeros(B, dtype=torch.float64, device=theta.device)
        grad = loglik_bwd(fctx.smc_ctx, theta, u, d, r, g_ell, g_sig2)
        return grad.to(fctx.in_dtype), None, None


def smc_get_particles(ctx: Context, theta=None, u=None, W=None):
    """Fill (or allocate on the context's device) theta [N,p], u [N,m] int32, W [N] float64.
    u=False skips the indices (returned as None)."""
    dev = ctx.device
    theta = theta if theta is not None else torch.empty(ctx.N, ctx.p, dtype=ctx.state_dtype,
                                                        device=dev)
    if u is False:
        u = None
    elif u is None:
        u = torch.empty(ctx.N, ctx.m, dtype=torch.int32, device=dev)
    W = W if W is not None else torch.empty(ctx.N, dtype=torch.float64, device=dev)
    check(_abi.load().smc_get_particles(ctx.handle, _ptr(theta), _ptr(u), _ptr(W)),
          "smc_get_particles", ctx.handle)
    return theta, u, W


def smc_set_particles(ctx: Context, theta, u, W=None) -> None:
    """Replace theta [N, p], u [N, m] and W [N] (each may be None: kept, W = 1/N); the cached
    estimates are recomputed."""
    theta = None if theta is None else theta.to(ctx.state_dtype).contiguous()
    u = None if u is None else u.to(torch.int32).contiguous()
    W = None if W is None else W.to(torch.float64).contiguous()
    check(_abi.load().smc_set_particles(ctx.handle, _ptr(theta), _ptr(u), _ptr(W)),
          "smc_set_particles", ctx.handle)


def smc_get_cache(ctx: Context):
    dev = ctx.device
    ell = torch.empty(ctx.N, dtype=torch.float64, device=dev)
    s2 = torch.empty_like(ell)
    blk = torch.empty(ctx.N, ctx.G, 2, dtype=torch.float64, device=dev)
    check(_abi.load().smc_get_cache(ctx.handle, _ptr(ell), _ptr(s2), _ptr(blk)), "smc_get_cache",
          ctx.handle)
    return ell, s2, blk


def smc_get_centre(ctx: Context):
    p = ctx.p
    tb, A, B, C = np.zeros(p), np.zeros(1), np.zeros(p), np.zeros((p, p))
    check(_abi.load().smc_get_centre(ctx.handle, _dp(tb), _dp(A), _dp(B), _dp(C)),
          "smc_get_centre", ctx.handle)
    return tb, float(A[0]), B, C


def smc_cv_moments(ctx: Context, theta):
    p = ctx.p
    th = np.ascontiguousarray(theta, dtype=np.float64)
    A, B, C = np.zeros(1), np.zeros(p), np.zeros((p, p))
    check(_abi.load().smc_cv_moments(ctx.handle, _dp(th), _dp(A), _dp(B), _dp(C)),
          "smc_cv_moments", ctx.handle)
    return float(A[0]), B, C


def smc_get_mass(ctx: Context):
    p = ctx.p
    S, L = np.zeros((p, p)), np.zeros((p, p))
    check(_abi.load().smc_get_mass(ctx.handle, _dp(S), _dp(L)), "smc_get_mass", ctx.handle)
    return S, L


def smc_get_status(ctx: Context) -> dict:
    a, lz, eps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    stage = ctypes.c_int32()
    check(_abi.load().smc_get_status(ctx.handle, ctypes.byref(a), ctypes.byref(lz),
                                     ctypes.byref(stage), ctypes.byref(eps)), "smc_get_status",
          ctx.handle)
    return {"a": a.value, "log_z": lz.value, "stage": stage.value, "eps": eps.value}


def smc_set_scalars(ctx: Context, stage: int, a: float, eps: float, log_z: float = 0.0) -> None:
    check(_abi.load().smc_set_scalars(ctx.handle, stage, a, eps, log_z), "smc_set_scalars",
          ctx.handle)


def smc_autotune(ctx: Context) -> tuple[int, int]:
    """Returns (estimator tile_hint, hmc_kernel) chosen by timing."""
    t, h = ctypes.c_int32(), ctypes.c_int32()
    check(_abi.load().smc_autotune(ctx.handle, ctypes.byref(t), ctypes.byref(h)), "smc_autotune",
          ctx.handle)
    return t.value, h.value


def smc_launch_count(ctx: Context) -> int:
    return int(_abi.load().smc_launch_count(ctx.handle))


PROFILE_GROUPS = ("estimate", "u_update", "hmc", "reweight", "moments_mass", "resample")


def smc_profile_enable(ctx: Context, on: bool = True) -> None:
    check(_abi.load().smc_profile_enable(ctx.handle, int(on)), "smc_profile_enable", ctx.handle)


def smc_profile_read(ctx: Context, group) -> tuple[int, float]:
    g = PROFILE_GROUPS.index(group) if isinstance(group, str) else int(group)
    n, ms = ctypes.c_int64(), ctypes.c_double()
    check(_abi.load().smc_profile_read(ctx.handle, g, ctypes.byref(n), ctypes.byref(ms)),
          "smc_profile_read", ctx.handle)
    return n.value, ms.value


# ------------------------------------------------------------------------------------------------
# Convenience wrapper
# ------------------------------------------------------------------------------------------------
def stage_log_line(rec: dict, status: dict) -> str:
    """One JSON line for a stage: the stage record (temperature, ESS, log-evidence increment,
    acceptance rates, moves) with the context's status after it (stage index, log Z, step)."""
    import json
    out = {"stage": int(status["stage"]), "a": float(rec["a"]), "ess": float(rec["ess"]),
           "log_z_inc": float(rec["log_z_inc"]), "log_z": float(status["log_z"]),
           "acc_u": float(rec["acc_u"]), "acc_theta": float(rec["acc_theta"]),
           "moves": int(rec["R"]), "eps": float(status["eps"])}
    return json.dumps(out)


class SubsampledSMC:
    """Likelihood-annealed subsampling SMC (Algorithm 2) on one GPU."""

    def __init__(self, X, y, family, prior_mean, prior_var, **kw):
        self.ctx = smc_init(X, y, family, prior_mean, prior_var, **kw)
        self.history = []

    def stage(self, R: int, adaptive=None) -> dict:
        """One stage with R moves, or with adaptive = (R_max, rho_max, quantile) the adaptive
        number of moves (smc_move_adaptive)."""
        a, lz, ess = smc_reweight(self.ctx)
        smc_resample(self.ctx)
        if adaptive is None:
            au, at = smc_move(self.ctx, R)
        else:
            R, au, at = smc_move_adaptive(self.ctx, *adaptive)
        rec = {"a": a, "log_z_inc": lz, "ess": ess, "acc_u": au, "acc_theta": at, "R": R}
        self.history.append(rec)
        return rec

    def run(self, R: int, max_stages: int = 1000, adaptive=None, log_path=None) -> dict:
        """Stages until a = 1. log_path: append one JSON line per stage (stage index, temperature,
        ESS, log-evidence increment and running total, acceptance rates, moves, step size)."""
        log = open(log_path, "a") if log_path else None
        try:
            while smc_get_status(self.ctx)["a"] < 1.0 and len(self.history) < max_stages:
                rec = self.stage(R, adaptive)
                if log is not None:
                    log.write(stage_log_line(rec, smc_get_status(self.ctx)) + "\n")
        finally:
            if log is not None:
                log.close()
        return smc_get_status(self.ctx)

    def particles(self):
        return smc_get_particles(self.ctx)

    def close(self):
        smc_free(self.ctx)


# ------------------------------------------------------------------------------------------------
# Particle shards (sharded.py combines them across processes)
# ------------------------------------------------------------------------------------------------
def smc_shard_export(ctx: Context, count: int):
    """This context's slice: theta [count, p], l_hat, sigma2_hat [count], blocks [count, G, 2]."""
    dev = ctx.device
    th = torch.empty(count, ctx.p, dtype=ctx.state_dtype, device=dev)
    ell = torch.empty(count, dtype=torch.float64, device=dev)
    s2 = torch.empty_like(ell)
    blk = torch.empty(count, ctx.G, 2, dtype=torch.float64, device=dev)
    check(_abi.load().smc_shard_export(ctx.handle, _ptr(th), _ptr(ell), _ptr(s2), _ptr(blk)),
          "smc_shard_export", ctx.handle)
    return th, ell, s2, blk


def smc_shard_import(ctx: Context, theta, ell, sigma2, blocks) -> None:
    """Overwrite theta [N, p] and the cached estimates of all N particles (no recomputation)."""
    th = theta.to(ctx.state_dtype).contiguous()
    e = ell.to(torch.float64).contiguous()
    s2 = sigma2.to(torch.float64).contiguous()
    b = blocks.to(torch.float64).contiguous()
    check(_abi.load().smc_shard_import(ctx.handle, _ptr(th), _ptr(e), _ptr(s2), _ptr(b)),
          "smc_shard_import", ctx.handle)


def smc_shard_gather_u(ctx: Context, idx: torch.Tensor, before_resample: bool) -> torch.Tensor:
    """u rows [len(idx), m] of global particles idx (before the last resampling if asked)."""
    idx = idx.to(device=ctx.device, dtype=torch.int32).contiguous()
    rows = torch.empty(idx.numel(), ctx.m, dtype=torch.int32, device=ctx.device)
    check(_abi.load().smc_shard_gather_u(ctx.handle, idx.numel(), _ptr(idx), _ptr(rows),
                                         int(bool(before_resample))),
          "smc_shard_gather_u", ctx.handle)
    return rows


def smc_shard_scatter_u(ctx: Context, idx: torch.Tensor, rows: torch.Tensor) -> None:
    idx = idx.to(device=ctx.device, dtype=torch.int32).contiguous()
    rows = rows.to(device=ctx.device, dtype=torch.int32).contiguous()
    check(_abi.load().smc_shard_scatter_u(ctx.handle, idx.numel(), _ptr(idx), _ptr(rows)),
          "smc_shard_scatter_u", ctx.handle)
    torch.cuda.current_stream(ctx.device).synchronize()  # idx and rows may be freed after return


def smc_move_accepts(ctx: Context) -> tuple[int, int]:
    au, at = ctypes.c_uint64(), ctypes.c_uint64()
    check(_abi.load().smc_move_accepts(ctx.handle, ctypes.byref(au), ctypes.byref(at)),
          "smc_move_accepts", ctx.handle)
    return au.value, at.value


def smc_finish_moves(ctx: Context, R: int, acc_u: int, acc_theta: int) -> None:
    check(_abi.load().smc_finish_moves(ctx.handle, int(R), int(acc_u), int(acc_theta)),
          "smc_finish_moves", ctx.handle)


def smc_resample_noalloc(W: torch.Tensor, seed: int, stage: int, ancestors: torch.Tensor,
                         stream=None) -> None:
    """Ancestors of systematic resampling without any device allocation by the library (for callers
    that cannot allocate, e.g. during CUDA graph capture). W: CUDA float64 [N], normalised;
    ancestors: CUDA int32 [N], written asynchronously on the stream. N <= 262144."""
    if W.dtype != torch.float64 or not W.is_cuda or not W.is_contiguous():
        raise ValueError("W must be a contiguous CUDA float64 tensor")
    if ancestors.dtype != torch.int32 or not ancestors.is_cuda or ancestors.numel() != W.numel():
        raise ValueError("ancestors must be a CUDA int32 tensor with W's length")
    with torch.cuda.device(W.device):
        rc = _abi.load().smc_resample_noalloc(W.numel(), _ptr(W), int(seed) & ((1 << 64) - 1),
                                              int(stage), _ptr(ancestors), _stream_handle(stream))
    check(rc, "smc_resample_noalloc", None)


# ------------------------------------------------------------------------------------------------
# Batches of independent posteriors
# ------------------------------------------------------------------------------------------------
class Batch:
    """Owns one smc_batch; `contexts` are its problems (for per-problem calls)."""

    def __init__(self, handle, contexts, keepalive):
        self.handle = handle
        self.contexts = contexts
        self._keepalive = keepalive

    def __del__(self):
        try:
            smc_batch_free(self)
        except Exception:
            pass


def _bcheck(code: int, where: str, handle) -> None:
    if code != 0:
        msg = _abi.load().smc_batch_last_error(handle)
        raise _abi.SmcError(code, where, (msg or b"").decode(errors="replace"))


def smc_batch_init(problems, stream=None) -> Batch:
    """problems: list of dicts with X, y, family, prior_mean, prior_var and the smc_init settings
    (N, m, G, L, seed; optional ess_frac, noise_sigma, dof, eps0, search_k, search_rounds,
    cv_order, cv_centre, resampling, grid_points, grid_decades, theta_move, hmc_kernel: 1 keeps
    the problem on the streamed trajectory kernel, 0 lets the batch pick a resident tile)."""
    lib = _abi.load()
    P = len(problems)
    probs = (SmcProblem * P)()
    cfgs = (SmcConfig * P)()
    keep = []
    meta = []
    for q, d in enumerate(problems):
        X = d["X"]
        if not X.is_cuda or X.dim() != 2 or X.stride(1) != 1 or X.dtype != torch.bfloat16:
            raise ValueError("batch problems need 2-D CUDA BF16 X with unit column stride")
        y = d["y"].to(device=X.device, dtype=torch.float32).contiguous()
        n, p = X.shape
        pm = np.ascontiguousarray(d["prior_mean"], dtype=np.float64)
        pv = np.ascontiguousarray(d["prior_var"], dtype=np.float64)
        probs[q] = SmcProblem(FAMILY[d["family"]], n, p, X.data_ptr(), DTYPE["bf16"], X.stride(0),
                              y.data_ptr(), _dp(pm), _dp(pv), float(d.get("noise_sigma", 1.0)),
                              float(d.get("dof", 5.0)))
        cfgs[q] = SmcConfig(d["N"], d["m"], d["G"], d["L"], float(d.get("ess_frac", 0.5)),
                            int(d["seed"]) & ((1 << 64) - 1), d.get("search_k", 16),
                            d.get("search_rounds", 10), float(d.get("eps0", 0.0)), 0,
                            int(d.get("hmc_kernel", 0)), 0,
                            int(d.get("cv_order", 2)), int(d.get("cv_centre", 0)), 0,
                            RESAMPLING[d.get("resampling", "systematic")],
                            int(d.get("grid_points", 0)), float(d.get("grid_decades", 0.0)),
                            THETA_MOVE[d.get("theta_move", "hmc")],
                            float(d.get("eps_jitter", 0.0)))
        keep += [y, pm, pv]
        meta.append((d["N"], d["m"], d["G"], p, n, X.device))
    handle = ctypes.c_void_p()
    with torch.cuda.device(meta[0][5]):
        rc = lib.smc_batch_init(ctypes.byref(handle), P, probs, cfgs, _stream_handle(stream))
    _bcheck(rc, "smc_batch_init", None)
    ctxs = []
    for q in range(P):
        h = ctypes.c_void_p()
        _bcheck(lib.smc_batch_context(handle, q, ctypes.byref(h)), "smc_batch_context", handle)
        N, m, G, p, n, dev = meta[q]
        ctxs.append(Context(h, N, m, G, p, n, torch.float32, dev, None, owned=False))
    return Batch(handle, ctxs, keep)


def smc_batch_free(b: Batch) -> None:
    if b.handle:
        for c in b.contexts:
            c.handle = ctypes.c_void_p()
        _abi.load().smc_batch_free(b.handle)
        b.handle = ctypes.c_void_p()


def smc_batch_stage(b: Batch, R: int, use_graph: bool = True) -> None:
    _bcheck(_abi.load().smc_batch_stage(b.handle, int(R), 1 if use_graph else 0),
            "smc_batch_stage", b.handle)


def smc_batch_autotune(b: Batch) -> int:
    t = ctypes.c_int32()
    _bcheck(_abi.load().smc_batch_autotune(b.handle, ctypes.byref(t)), "smc_batch_autotune",
            b.handle)
    return t.value


def smc_batch_tile(b: Batch) -> int:
    t = ctypes.c_int32()
    _bcheck(_abi.load().smc_batch_tile(b.handle, ctypes.byref(t)), "smc_batch_tile", b.handle)
    return t.value


def smc_batch_hmc_kernel(b: Batch, q: int) -> int:
    """Problem q's trajectory kernel as an hmc_kernel value (1 streamed, k >= 2 resident tile)."""
    t = ctypes.c_int32()
    _bcheck(_abi.load().smc_batch_hmc_kernel(b.handle, int(q), ctypes.byref(t)),
            "smc_batch_hmc_kernel", b.handle)
    return t.value


def smc_batch_launch_count(b: Batch) -> int:
    return int(_abi.load().smc_batch_launch_count(b.handle))


def smc_batch_context(b: Batch, q: int) -> Context:
    """The context of problem q (owned by the batch)."""
    return b.contexts[q]


def smc_batch_last_error(b: Batch | None = None) -> str:
    msg = _abi.load().smc_batch_last_error(b.handle if b is not None else None)
    return (msg or b"").decode(errors="replace")
