#!/usr/bin/env python
"""Benchmark of likelihood-annealed subsampling SMC on one GB300 (or N replicas under torchrun).

A step is one complete SMC run of the workload (Algorithm 2 to completion): smc_init (packing X,
the posterior-mode centre by Newton's method, the control-variate moments A, B, C, initial
particles and their cached estimates), then stages of temperature search + reweighting, weighted
moments + mass matrix, systematic resampling and R Markov moves (Algorithm 1: block u update, then
an HMC trajectory of L leapfrog steps) until the temperature reaches 1, and the posterior (weighted
mean, log Z) read back. The metric is particle-row gradient evaluations per second over whole
runs: each stage evaluates the subsampled log-likelihood gradient N * m * R * (L + 1) times;
ms_per_step is the SMC wall time from initialisation to a = 1.

Default workload: logistic regression, n = 1,000,000 rows, p = 20 (intercept + 19 AR(1) N(0,1)
covariates), N = 4096 particles, m = 1000, G = 10, L = 20, R = 5, X stored in BF16 with FP32
accumulation (the FP32-stored run is measured beside it). Data are synthetic (seeded).

--impl reference times the FP64 CPU oracle on the host cores instead (bounded particle samples).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

R_MOVES = 5
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 80.6: SMs x FP32 lanes x FMA x max SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-compare", action="store_true", help="skip the FP32-stored comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--no-gather", action="store_true",
                    help="skip the HBM-bound gather leg (Poisson n=5e6, p=50)")
    ap.add_argument("--gather-only", action="store_true",
                    help="run only the HBM-bound gather leg and print its JSON (for profiling)")
    ap.add_argument("--gather-tile", type=int, default=0,
                    help="estimator tile hint for the gather leg (0: autotune)")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph stage timing")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched uneven-posteriors leg (64 problems)")
    ap.add_argument("--no-full", action="store_true",
                    help="skip the full-data comparison leg (about 5 s)")
    ap.add_argument("--no-gam", action="store_true",
                    help="skip the GAM gather leg (n=1e7, p=101; about 10-30 s of data generation)")
    ap.add_argument("--gam-n", type=int, default=10_000_000,
                    help="rows of the GAM workload (smaller for profiling captures)")
    ap.add_argument("--gam-only", action="store_true",
                    help="run only the GAM gather leg and print its JSON (for profiling)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched-posteriors leg and print its JSON (for profiling)")
    ap.add_argument("--profile-stages", type=int, default=0,
                    help="run only the first K stages of one run of the default workload with the "
                         "default kernels (no autotune), for ncu captures of a chosen stage")
    ap.add_argument("--hmc-kernel", type=int, default=0,
                    help="with --profile-stages: the trajectory kernel (smc_config.hmc_kernel)")
    return ap.parse_args()


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload_name(wl, R):
    return (f"logistic n={wl.n} p={wl.p} N={wl.N} m={wl.m} G={wl.G} L={wl.L} R={R} "
            f"X={wl.x_dtype}")


METRIC = "particle-row grad-evals/s (complete subsampling SMC runs, init to a = 1)"


def bench_config(wl, R, world):
    """The config object of both arms' JSON lines (the same workload and step definition)."""
    return {"workload": workload_name(wl, R), "model": "logistic regression",
            "global_batch": wl.N * world, "seq_len": wl.m, "parallelism": f"replicas{world}",
            "stage_window": "complete runs: every stage from initialisation to a = 1",
            "l2": "flushed between timed runs (256 MiB write)",
            "accumulate": "FP32 per row, FP64 totals/weights/MH"}


STEP = ("one complete SMC run: smc_init (packing, Newton centre, A/B/C, initial particles and "
        "cache) + every stage to a = 1 + the posterior read back")


def grad_evals_per_stage(wl, R):
    return wl.N * wl.m * R * (wl.L + 1)


# ------------------------------------------------------------------------------------------------
# Clock sampling during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.reader.join(timeout=2)
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def device_workload(wl, dev):
    import torch
    if wl.x_dtype == "bf16":
        X = torch.from_numpy(wl.X_store.view(np.int16)).view(torch.bfloat16)
    else:
        X = torch.from_numpy(wl.X_store)
    return X.to(dev), torch.from_numpy(wl.y_store).to(dev)


def make_ctx(S, wl, dev, seed_offset=0, **kw):
    X, y = device_workload(wl, dev)
    args = dict(ess_frac=0.5, theta_bar=None, noise_sigma=wl.sigma, dof=wl.dof)
    args.update(kw)
    ctx = S.smc_init(X, y, wl.family, wl.prior_mean, wl.prior_var, N=wl.N, m=wl.m, G=wl.G, L=wl.L,
                     seed=wl.seed + seed_offset, **args)
    del X, y  # the library keeps its own packed copy
    tile = S.smc_autotune(ctx)
    return ctx, tile


def run_stage(S, ctx, R):
    a, lz, ess = S.smc_reweight(ctx)
    S.smc_resample(ctx)
    S.smc_move(ctx, R)
    return a


def max_over_ranks(value: float, device) -> float:
    """The largest of every rank's value (the timing rule: the job's time is its slowest rank)."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_step: float, steps: int, world: int, ms: float) -> float:
    """Whole-job throughput: every rank processes units_per_step per step (replicas, weak scaling);
    ms is the slowest rank's time for the steps."""
    return units_per_step * steps * world / (ms / 1e3)


def complete_run(S, wl, Xd, yd, R, hints, seed, profile=False, max_stages=400, host_out=None):
    """One benchmark step: a complete SMC run (init to a = 1) on the resident inputs Xd, yd, ending
    with the posterior read back: the weighted mean of theta (device reduction, p values to the
    host) and log Z; with host_out = (theta_h, W_h) pinned buffers, the whole weighted cloud is
    copied to the host instead. hints: the (tile_hint, hmc_kernel) the autotuner chose. Returns
    the context (still open: freed by the caller outside the timed region), stages, log Z and the
    posterior mean."""
    ctx = S.smc_init(Xd, yd, wl.family, wl.prior_mean, wl.prior_var, N=wl.N, m=wl.m, G=wl.G,
                     L=wl.L, seed=seed, ess_frac=0.5, theta_bar=None, noise_sigma=wl.sigma,
                     dof=wl.dof, tile_hint=hints[0], hmc_kernel=hints[1])
    if profile:
        S.smc_profile_enable(ctx, True)
    stages, a = 0, 0.0
    while a < 1.0 and stages < max_stages:
        a = run_stage(S, ctx, R)
        stages += 1
    if host_out is None:
        th, _, W = S.smc_get_particles(ctx, u=False)
        mean = (th.double() * W[:, None]).sum(0).cpu().numpy()
    else:
        th_h, W_h = host_out
        S.smc_get_particles(ctx, th_h, False, W_h)
        mean = (th_h.double() * W_h[:, None]).sum(0).numpy()
    lz = S.smc_get_status(ctx)["log_z"]
    return ctx, stages, lz, mean


def timed_runs(S, wl, Xd, yd, R, hints, steps, warmup, flush, dist, seed):
    """`warmup` untimed complete runs, then `steps` timed ones (CUDA events on the library's
    stream around each run; the L2 flush before each). Per-kernel-group device times come from the
    library's tracing events over the timed runs."""
    import torch
    for _ in range(warmup):
        ctx, _, _, _ = complete_run(S, wl, Xd, yd, R, hints, seed)
        S.smc_free(ctx)
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    ms, stages, launches, lzs = [], [], 0, []
    prof = {g: [0, 0.0] for g in S.smc.PROFILE_GROUPS}
    t0 = time.perf_counter()
    for _ in range(steps):
        flush.add_(1)  # write a buffer larger than L2 between timed runs
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx, k, lz, _ = complete_run(S, wl, Xd, yd, R, hints, seed, profile=True)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        stages.append(k)
        lzs.append(lz)
        launches += S.smc_launch_count(ctx)
        for g in S.smc.PROFILE_GROUPS:
            n_g, t_g = S.smc_profile_read(ctx, g)
            prof[g][0] += n_g
            prof[g][1] += t_g
        S.smc_free(ctx)
    wall = time.perf_counter() - t0
    tot = sum(ms)
    if dist:
        tot = max_over_ranks(tot, "cuda")
    return tot, wall, launches, prof, stages, lzs


def hmc_by_stage(S, ctx, R, max_stages=400):
    """Device time of the HMC trajectory launch at every stage of one complete run (the kernel's
    cost depends on how far the particles are from the centre), with the stage's temperature."""
    S.smc_profile_enable(ctx, True)
    S.smc_profile_read(ctx, "hmc")
    out, a = [], 0.0
    while a < 1.0 and len(out) < max_stages:
        a = run_stage(S, ctx, R)
        n_h, t_h = S.smc_profile_read(ctx, "hmc")
        out.append([round(a, 8), round(t_h / max(n_h, 1), 4)])
    S.smc_profile_enable(ctx, False)
    return out


def full_run(S, wl, dev, R, max_stages=400, adaptive=None, **kw):
    """SMC wall time from init to a = 1 (Algorithm 2 to completion). kw: smc_init options (the
    paper's stage settings); adaptive: (R_max, rho_max, quantile) for the adaptive move count."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx, _ = make_ctx(S, wl, dev, seed_offset=1000, **kw)
    stages = 0
    moves = 0
    a = 0.0
    while a < 1.0 and stages < max_stages:
        a, _, _ = S.smc_reweight(ctx)
        S.smc_resample(ctx)
        if adaptive is None:
            S.smc_move(ctx, R)
            moves += R
        else:
            moves += S.smc_move_adaptive(ctx, *adaptive)[0]
        stages += 1
    th, _, W = S.smc_get_particles(ctx)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = S.smc_get_status(ctx)
    mean = (th.double() * W[:, None]).sum(0).cpu().numpy()
    tb = S.smc_get_centre(ctx)[0]
    S.smc_free(ctx)
    return {"wall_s": round(wall, 4), "stages": stages, "moves": moves, "log_z": st["log_z"],
            "post_mean_minus_centre_maxabs": float(np.max(np.abs(mean - tb)))}


def gather_leg(S, dev, hbm, wl=None, reps=20, stages=3, tile_hint=0):
    """HBM-bound leg. Default workload: Poisson regression, n = 5e6, p = 50, BF16 X (640 MB packed,
    far above L2), N = 8192, m = 2000 (the GAM workload, n = 1e7, p = 101, is the other one). Times
    the subsampled estimator with gradient over all particles (one gather of N*m rows per call, the
    streamed kernel; X is larger than L2, so no flush is needed between calls) and a few full SMC
    stages, whose rows per particle do not fit in shared memory (streamed HMC kernel)."""
    import torch
    if wl is None:
        from smc_workloads import poisson_5e6
        wl = poisson_5e6("bf16", upcast=False)
    X, y = device_workload(wl, dev)
    ctx = S.smc_init(X, y, wl.family, wl.prior_mean, wl.prior_var, N=wl.N, m=wl.m, G=wl.G,
                     L=wl.L, seed=wl.seed, ess_frac=0.5, theta_bar=None, tile_hint=tile_hint,
                     noise_sigma=wl.sigma)
    del X, y
    tile = S.smc_autotune(ctx) if tile_hint == 0 else (tile_hint, 1)
    theta, u, _ = S.smc_get_particles(ctx)
    for _ in range(3):
        S.loglik_grad(ctx, theta, u, 1.0)
    S.smc_profile_enable(ctx, True)
    S.smc_profile_read(ctx, "estimate")
    for _ in range(reps):
        S.loglik_grad(ctx, theta, u, 1.0)
    n_e, ms_e = S.smc_profile_read(ctx, "estimate")
    bytes_row = wl.p * 2 + 4 + 4
    bytes_call = wl.N * wl.m * bytes_row
    per_call = ms_e / max(n_e, 1)
    for g in S.smc.PROFILE_GROUPS:
        S.smc_profile_read(ctx, g)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(stages)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(stages)]
    for k in range(stages):
        starts[k].record()
        run_stage(S, ctx, wl.R)
        ends[k].record()
    torch.cuda.synchronize()
    ms_stage = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / stages
    n_h, ms_h = S.smc_profile_read(ctx, "hmc")
    S.smc_profile_enable(ctx, False)
    S.smc_free(ctx)
    achieved = bytes_call / (per_call / 1e3) / 1e9
    hmc_bytes = (wl.L + 1) * bytes_call
    esz = 2
    row_b = ((wl.p * esz + 15) // 16 * 16 + 16 + 63) // 64 * 64
    return {"workload": f"{wl.family} n={wl.n} p={wl.p} N={wl.N} m={wl.m} G={wl.G} L={wl.L} "
                        f"R={wl.R} X=bf16 (packed X {wl.n * row_b / 1e6:.0f} MB > L2)",
            "tile": tile,
            "estimator": {"kernel": "k_estimate (loglik_grad over all particles)",
                          "ms_per_call": per_call, "bytes_per_call": bytes_call,
                          "achieved_gbs": achieved, "frac_of_hbm": achieved / hbm,
                          "grad_evals_per_s": wl.N * wl.m / (per_call / 1e3)},
            "stage": {"ms_per_stage": ms_stage,
                      "grad_evals_per_s": wl.N * wl.m * wl.R * (wl.L + 1) / (ms_stage / 1e3),
                      "hmc_ms_per_launch": ms_h / max(n_h, 1),
                      "hmc_achieved_gbs": hmc_bytes / (ms_h / max(n_h, 1) / 1e3) / 1e9}}


def full_data_leg(S, wl, dev, R, tc_peak, stages=2, reps=5):
    """The comparison method (full-data SMC, exact log-likelihood) on the same workload: one
    loglik_full evaluation over all N particles x n rows (the tcgen05 kernel), and `stages` full
    SMC stages (reweight, resample, R HMC moves with L + 1 full-data evaluations each)."""
    import torch
    X, y = device_workload(wl, dev)
    ctx = S.smc_init(X, y, wl.family, wl.prior_mean, wl.prior_var, N=wl.N, m=1, G=1, L=wl.L,
                     seed=wl.seed, ess_frac=0.5, theta_bar=None, full_data=True)
    del X, y
    th, _, _ = S.smc_get_particles(ctx)
    for _ in range(2):
        S.loglik_full(ctx, th, 1.0)
    S.smc_profile_enable(ctx, True)
    S.smc_profile_read(ctx, "estimate")
    for _ in range(reps):
        S.loglik_full(ctx, th, 1.0)
    n_e, ms_e = S.smc_profile_read(ctx, "estimate")
    per_eval = ms_e / max(n_e, 1)
    S.smc_profile_enable(ctx, False)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(stages):
        run_stage(S, ctx, R)
    t1.record()
    torch.cuda.synchronize()
    ms_stage = t0.elapsed_time(t1) / stages
    S.smc_free(ctx)
    kp = (wl.p + 15) // 16 * 16
    mma_flops = 2.0 * wl.N * wl.n * kp * (3 + 2)  # GEMM1: 3 theta terms; GEMM2: 2 l' terms
    return {"kernel": "k_full_mma (eta = Theta X', family terms, l' X on tcgen05)",
            "ms_per_eval": per_eval,
            "particle_rows_per_s": wl.N * wl.n / (per_eval / 1e3),
            "tensor_tflops": mma_flops / (per_eval / 1e3) / 1e12,
            "tensor_peak_tflops": tc_peak,
            "ms_per_stage": ms_stage,
            "grad_evals_per_s": wl.N * wl.n * R * (wl.L + 1) / (ms_stage / 1e3),
            "note": "bound by the per-element family terms (3 MUFU ops per particle-row), not the "
                    "MMAs"}


def precision_leg(S, dev, R=5, seeds=3, n=1_000_000, p=20, max_stages=400):
    """Mixed precision against FP32 storage at equal accuracy: a conjugate Gaussian linear model of
    the headline shape (n = 1e6, p = 20, N = 4096, m = 1000, L = 20; sigma = 0.5, prior N(0, 10 I)),
    where the second-order control variate is exact, so each storage type has a closed-form
    posterior mean and log marginal likelihood on its own stored values. Complete SMC runs
    (init to a = 1) in BF16 and FP32 storage, timed, with their errors against those closed forms
    (several seeds: the errors are Monte Carlo error)."""
    import torch
    from smc_workloads import small_glm
    out = {}
    for x_dtype in ("bf16", "f32"):
        wl = small_glm("gaussian", n=n, p=p, N=4096, m=1000, G=10, L=20, R=R, x_dtype=x_dtype,
                       seed=11, sigma=0.5, theta_scale=0.3, prior_var=10.0)
        X, y, s2, tau2 = wl.X, wl.y, wl.sigma ** 2, 10.0
        XtX = X.T @ X
        Sinv = XtX / s2 + np.eye(p) / tau2
        mu = np.linalg.solve(Sinv, X.T @ y / s2)
        sd = np.sqrt(np.diag(np.linalg.inv(Sinv)))
        logdet = np.linalg.slogdet(np.eye(p) + tau2 * XtX / s2)[1]
        logml = (-0.5 * n * math.log(2 * math.pi * s2) - 0.5 * logdet
                 - (y @ y - y @ X @ mu) / (2 * s2))
        walls, lz_err, mean_err, stages = [], [], [], []
        for s in range(seeds):
            Xd, yd = device_workload(wl, dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx = S.smc_init(Xd, yd, "gaussian", wl.prior_mean, wl.prior_var, N=wl.N, m=wl.m,
                             G=wl.G, L=wl.L, seed=100 + s, ess_frac=0.5, noise_sigma=wl.sigma,
                             theta_bar=None)
            k, a = 0, 0.0
            while a < 1.0 and k < max_stages:
                a = run_stage(S, ctx, R)
                k += 1
            th, _, W = S.smc_get_particles(ctx)
            mean = (th.double() * W[:, None]).sum(0).cpu().numpy()
            torch.cuda.synchronize()
            walls.append(time.perf_counter() - t0)
            lz_err.append(S.smc_get_status(ctx)["log_z"] - logml)
            mean_err.append(float(np.max(np.abs(mean - mu) / sd)))
            stages.append(k)
            S.smc_free(ctx)
            del Xd, yd
        out[x_dtype] = {"wall_s_mean": float(np.mean(walls)), "stages": stages,
                        "log_z_minus_closed_form": [round(e, 4) for e in lz_err],
                        "post_mean_err_max_sd": [round(e, 4) for e in mean_err]}
    out["bf16_speedup"] = out["f32"]["wall_s_mean"] / out["bf16"]["wall_s_mean"]
    out["workload"] = (f"gaussian n={n} p={p} N=4096 m=1000 G=10 L=20 R={R}, sigma=0.5, "
                       f"prior N(0,10I); wall time includes init (packing, Newton centre)")
    return out


def student_t_leg(S, dev, R=5, max_stages=200, N=280, seeds=3):
    """Sec. 4.3's Student-t comparison in the paper's shape (n = 5e5, p = 50 correlated
    covariates, t_5 errors, m = 1250, G = 100; the paper's M = 280 particles, L = 20, BF16 X):
    complete SMC runs (init to a = 1) with subsampling and with the full-data method, on the same
    GPU, over a few seeds (the paper reports means and standard errors over 10 runs, and the
    subsampling approach 6.5 to 10.5 times faster on its CPU cluster, Table 3)."""
    import torch
    from smc_workloads import student_t_5e5
    wl = student_t_5e5("bf16", N=N)
    res = {}
    for full in (False, True):
        walls, lzs, nst = [], [], []
        for s in range(seeds):
            X, y = device_workload(wl, dev)
            ctx = S.smc_init(X, y, "student_t", wl.prior_mean, wl.prior_var, N=wl.N,
                             m=1 if full else wl.m, G=1 if full else wl.G, L=wl.L,
                             seed=wl.seed + 1000 * s, ess_frac=0.5, noise_sigma=wl.sigma,
                             dof=wl.dof, theta_bar=None, full_data=full)
            del X, y
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            stages, a = 0, 0.0
            while a < 1.0 and stages < max_stages:
                a = run_stage(S, ctx, R)
                stages += 1
            torch.cuda.synchronize()
            walls.append(time.perf_counter() - t0)
            lzs.append(S.smc_get_status(ctx)["log_z"])
            nst.append(stages)
            S.smc_free(ctx)
        res["full_data" if full else "subsampling"] = {
            "wall_s_mean": round(float(np.mean(walls)), 4), "stages": nst,
            "log_z_mean": float(np.mean(lzs)),
            "log_z_se": float(np.std(lzs, ddof=1) / math.sqrt(seeds)) if seeds > 1 else None,
            "ms_per_stage": float(np.mean(walls)) * 1e3 / float(np.mean(nst))}
    res["speedup_wall"] = res["full_data"]["wall_s_mean"] / res["subsampling"]["wall_s_mean"]
    res["log_z_diff"] = res["subsampling"]["log_z_mean"] - res["full_data"]["log_z_mean"]
    res["workload"] = (f"{wl.name} N={wl.N} m={wl.m} G={wl.G} L={wl.L} R={R}, "
                       "ESS target 0.5N, centre = posterior mode")
    return res


def batch_leg(S, dev, P=64, stages=5, warmup=3):
    """Batched uneven posteriors: 64 logistic/probit problems (n log-uniform in [1e4, 1e6], p in
    5..40, N = 1024 each, m = clamp(ceil(n/1000), 100, 1000), G = 10, L = 20, R = 5): the stage
    steps of all problems in shared launches, per move one u-update launch over all particles and
    one trajectory launch per tile group; timed as graph-replayed stages and launch by launch;
    estimator tile from the batch autotuner."""
    import torch
    from smc_workloads import batch_uneven
    t0 = time.perf_counter()
    wls = batch_uneven(P=P, upcast=False)
    gen_s = time.perf_counter() - t0
    probs = []
    for w in wls:
        X, y = device_workload(w, dev)
        probs.append(dict(X=X, y=y, family=w.family, prior_mean=w.prior_mean,
                          prior_var=w.prior_var, N=w.N, m=w.m, G=w.G, L=w.L, seed=w.seed))
    b = S.smc_batch_init(probs)
    del probs
    tile = S.smc_batch_autotune(b)
    R = wls[0].R
    per_stage = sum(w.N * w.m for w in wls) * R * (wls[0].L + 1)
    out = {"workload": f"{P} problems: logistic/probit, n log-uniform [1e4, 1e6] "
                       f"(total {sum(w.n for w in wls)} rows), p 5..40, N=1024 each, "
                       f"m=clamp(n/1000,100,1000), G=10, L=20, R=5, X=bf16",
           "tile": tile, "data_generation_s": round(gen_s, 1)}
    for name, graph in (("graph", True), ("launches", False)):
        for _ in range(warmup):
            S.smc_batch_stage(b, R, use_graph=graph)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = S.smc_batch_launch_count(b)
        e0.record()
        for _ in range(stages):
            S.smc_batch_stage(b, R, use_graph=graph)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / stages
        out[name] = {"ms_per_stage": ms, "grad_evals_per_s": per_stage / (ms / 1e3),
                     "launches_per_stage": (S.smc_batch_launch_count(b) - l0) / stages}
    S.smc_batch_free(b)
    return out


def gam_leg(S, dev, hbm, tile_hint=0, n=10_000_000):
    """The GAM workload (Gaussian response, sigma = 0.5, n = 1e7, p = 101 B-spline columns, BF16;
    N = 16384, m = 5000, L = 25) through the gather leg: 82M gathered rows per estimator call."""
    from smc_workloads import gam_1e7
    t0 = time.perf_counter()
    wl = gam_1e7("bf16", n=n, upcast=False)
    gen_s = time.perf_counter() - t0
    out = gather_leg(S, dev, hbm, wl=wl, reps=10, stages=1, tile_hint=tile_hint)
    out["data_generation_s"] = round(gen_s, 1)
    return out


def e2e_runs(S, wl, R, hints, steps, dev, seed):
    """The same complete runs through the public API with the inputs in pinned host memory: each
    step copies X and y to the device, runs init to a = 1, and copies the weighted cloud (theta,
    W) back to pinned host memory with log Z."""
    import torch
    if wl.x_dtype == "bf16":
        X_h = torch.from_numpy(wl.X_store.view(np.int16)).view(torch.bfloat16).pin_memory()
    else:
        X_h = torch.from_numpy(wl.X_store).pin_memory()
    y_h = torch.from_numpy(wl.y_store).pin_memory()
    th_h = torch.empty(wl.N, wl.p, dtype=torch.float32).pin_memory()
    W_h = torch.empty(wl.N, dtype=torch.float64).pin_memory()
    bytes_in = X_h.numel() * X_h.element_size() + y_h.numel() * y_h.element_size()
    bytes_out = th_h.numel() * 4 + W_h.numel() * 8 + 8
    units = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        Xd = X_h.to(dev, non_blocking=True)
        yd = y_h.to(dev, non_blocking=True)
        ctx, k, _, _ = complete_run(S, wl, Xd, yd, R, hints, seed, host_out=(th_h, W_h))
        units += k * grad_evals_per_stage(wl, R)
        S.smc_free(ctx)
        del Xd, yd
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return units / wall, bytes_in, bytes_out


def graph_stage_leg(S, wl, dev, R, hints, seed):
    """The stages of one complete run (after init) replayed as captured CUDA graphs (smc_stage,
    no host synchronisation inside a stage) against the same stages launched one by one."""
    import torch
    out = {}
    Xd, yd = device_workload(wl, dev)
    for name, graph in (("launches", False), ("graph", True)):
        ctx = S.smc_init(Xd, yd, wl.family, wl.prior_mean, wl.prior_var, N=wl.N, m=wl.m, G=wl.G,
                         L=wl.L, seed=seed, ess_frac=0.5, theta_bar=None, tile_hint=hints[0],
                         hmc_kernel=hints[1])
        torch.cuda.synchronize()
        l0 = S.smc_launch_count(ctx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        k, a = 0, 0.0
        while a < 1.0 and k < 400:
            if graph:
                S.smc_stage(ctx, R, use_graph=True)
                a = S.smc_get_status(ctx)["a"]
            else:
                a = run_stage(S, ctx, R)
            k += 1
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"stages": k, "ms_per_stage": ms / k,
                     "grad_evals_per_s": k * grad_evals_per_stage(wl, R) / (ms / 1e3),
                     "launches_per_stage": (S.smc_launch_count(ctx) - l0) / k}
        S.smc_free(ctx)
    out["note"] = ("stages of one run (init excluded); graph: one smc_stage graph launch per "
                   "stage (the first two stages capture) and one status read")
    return out


def gpu_arm(args):
    import torch
    import paper_1805_03317_gb300 as S
    from smc_workloads import logistic_1e6

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    R = R_MOVES
    wl = logistic_1e6("bf16", n=args.n)
    seed = wl.seed + rank  # replicas: each rank runs its own chain

    # the estimator tile and trajectory kernel, chosen once by the library's autotuner on this
    # workload (untimed) and passed to every timed run as hints; then the per-stage profile of
    # one complete run
    ctx0, hints = make_ctx(S, wl, dev, seed_offset=rank)
    by_stage = hmc_by_stage(S, ctx0, R)
    S.smc_free(ctx0)

    Xd, yd = device_workload(wl, dev)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2
    sampler = ClockSampler(local if not os.environ.get("CUDA_VISIBLE_DEVICES") else 0)
    sampler.start()
    ms, wall, launches, prof, stages, lzs = timed_runs(S, wl, Xd, yd, R, hints, args.steps,
                                                       args.warmup, flush, dist, seed)
    clocks = sampler.stop()
    del Xd, yd
    units = sum(stages) * grad_evals_per_stage(wl, R)
    value = units * world / (ms / 1e3)

    # roofline of the dominant kernel, the HMC trajectory with the subsample resident in shared
    # memory. It reads X once per trajectory and then runs L+1 estimator passes out of shared
    # memory, so it is bound by the FP32/integer issue rate, not by HBM: bound "alu" against the
    # FP32 peak 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz. Algorithmic FLOPs per particle-row
    # evaluation: 8p, the four length-p products of a row (x'theta, x'theta_bar, sum r x,
    # sum d r x); the second is cached per row here, but the count keeps it.
    hbm, peak_kind = peaks()
    n_h, ms_h = prof["hmc"]
    units_launch = (wl.L + 1) * wl.N * wl.m
    flops_launch = units_launch * 8 * wl.p
    sec = ms_h / max(n_h, 1) / 1e3
    achieved = flops_launch / sec / 1e12 if n_h else None
    bytes_row = wl.p * 2 + 4 + 4
    bytes_launch = units_launch * bytes_row
    shares = {g: round(v[1] / ms, 4) for g, v in prof.items() if v[0]}

    e2e_value, bi, bo = e2e_runs(S, wl, R, hints, args.steps, dev, seed)

    graph = None
    if not args.no_graph:
        graph = graph_stage_leg(S, wl, dev, R, hints, seed)

    fp32 = None
    walls = {}
    if not args.no_compare and rank == 0:
        wl32 = logistic_1e6("f32", n=args.n)
        c32, hints32 = make_ctx(S, wl32, dev, seed_offset=rank)
        S.smc_free(c32)
        X32, y32 = device_workload(wl32, dev)
        ms32, _, _, prof32, st32, lz32 = timed_runs(S, wl32, X32, y32, R, hints32, args.steps,
                                                    args.warmup, flush, False, seed)
        del X32, y32
        n32, t32 = prof32["hmc"]
        fp32 = {"value": sum(st32) * grad_evals_per_stage(wl32, R) / (ms32 / 1e3),
                "ms_per_step": ms32 / args.steps, "stages_per_run": sorted(set(st32)),
                "log_z": lz32[0], "hmc_ms_per_launch": t32 / max(n32, 1), "tile": hints32,
                "bf16_speedup_wall": (ms32 / args.steps) / (ms / args.steps)}
        del wl32
        # the paper's own stage settings (Algorithm 2 as printed): ESS target 0.8N by the grid
        # rule, multinomial resampling, control variates re-centred every stage, R tuned per stage
        # R = 10 moves per stage on the conjugate leg: at p = 20 the five moves of the workload
        # leave the cloud short of the tempered target each stage and log Z about 0.2 low (FP64
        # oracle: -0.18 mean over four seeds at R = 5, -0.05 at R = 10, n = 2e4, N = 4096)
        walls["conjugate_bf16_vs_fp32"] = precision_leg(S, dev, 10)
        walls["bf16_paper_settings"] = full_run(
            S, wl, dev, R, adaptive=(30, 0.1, 0.9), ess_frac=0.8, grid_points=1024,
            resampling="multinomial", cv_centre=1)

    full = None
    tleg = None
    if not args.no_full and rank == 0:
        full = full_data_leg(S, wl, dev, R, bf16_peak())
        full["subsampling_speedup_per_stage"] = full["ms_per_stage"] / (ms / sum(stages))
        tleg = student_t_leg(S, dev, R)

    batch = None
    if not args.no_batch and rank == 0:
        batch = batch_leg(S, dev)

    gather = None
    if not args.no_gather and rank == 0:
        gather = gather_leg(S, dev, hbm)
    gam = None
    if not args.no_gam and rank == 0:
        gam = gam_leg(S, dev, hbm, n=args.gam_n)

    cpu = None
    if not args.no_cpu and rank == 0:
        cpu = cpu_baseline(wl, R, args.cpu_seconds)

    traffic = committed_traffic(bytes_launch)
    config = bench_config(wl, R, world)
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "grad-evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16",
        "data": "synthetic",
        "config": config,
        "step": STEP,
        "stages_per_run": sorted(set(stages)),
        "tile": list(hints),
        "roofline": {"kernel": "k_hmc_res (HMC trajectory, rows resident in shared memory)",
                     "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                     "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                     "unit": "TFLOP/s", "frac": (achieved / FP32_PEAK_TFLOPS) if achieved else None,
                     "traffic": traffic, "flops_per_launch": flops_launch,
                     "flops_per_unit": 8 * wl.p,
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "algorithmic_gbs": bytes_launch / sec / 1e9 if n_h else None,
                     "hbm_peak_gbs": hbm, "hbm_peak_kind": peak_kind,
                     "launches": n_h, "ms_per_launch": ms_h / max(n_h, 1),
                     "note": "averaged over every HMC launch of the timed runs (all stages); "
                             "traffic = DRAM bytes per launch (ncu); the rows of a particle are "
                             "gathered once per trajectory, the L+1 passes read shared memory"},
        "hmc_ms_by_stage": by_stage,
        "stage_shares": shares,
        "log_z": lzs[0] if lzs else None,
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": "grad-evals/s", "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo},
        "fp32_storage": fp32,
        "graph_stages": graph,
        "full_data_comparison": full,
        "student_t_comparison": tleg,
        "batched_posteriors": batch,
        "hbm_gather_leg": gather,
        "gam_gather_leg": gam,
        "smc_wall_time": walls,
        "cpu_baseline": cpu,
        "wall_s_timed": wall,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def committed_traffic(bytes_launch):
    """DRAM bytes per HMC launch from the committed ncu summary, if it was taken on the current
    kernel sources (its recorded source hash matches); otherwise None."""
    path = os.path.join(ROOT, "profiles", "k_hmc_res_logistic_n1e6_p20_bf16.txt")
    try:
        text = open(path).read()
    except OSError:
        return None
    want = source_hash()
    vals = {}
    for line in text.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("csrc_sha256") != want or "dram_bytes_per_launch_full" not in vals:
        return None
    try:
        return float(vals["dram_bytes_per_launch_full"])
    except ValueError:
        return None


def source_hash():
    """Hash of the sources that define the HMC trajectory kernels for BF16 storage."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1805_03317_gb300", "csrc")
    for f in ("device.cuh", "estimator.cuh", "resident.cuh", "res_bf16.cu", "internal.h"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ------------------------------------------------------------------------------------------------
def oracle_setup(wl):
    from oracle import oracle as O
    prob = O.Problem(wl.family, wl.X, wl.y, wl.prior_mean, wl.prior_var)
    prob.set_centre(wl.theta_true)  # the oracle's own move timing does not depend on the centre
    th, us = O.init_particles(wl.seed, wl.N, wl.p, wl.m, wl.n, wl.prior_mean, wl.prior_var)
    Sig = np.diag(wl.prior_var)
    Lc = np.linalg.cholesky(Sig)
    return O, prob, th, us, Sig, Lc


def oracle_move_seconds(O, prob, wl, th, us, Sig, Lc, count, stage):
    t0 = time.perf_counter()
    O.upm_move(prob, wl.m, wl.G, wl.seed, stage, 0, 0.01, th[:count], us[:count])
    O.hmc_move(prob, wl.m, wl.G, wl.seed, stage, 0, 0.01, 0.3, wl.L, Sig, Lc, th[:count],
               us[:count])
    return time.perf_counter() - t0


def cpu_baseline(wl, R, seconds):
    O, prob, th, us, Sig, Lc = oracle_setup(wl)
    cores = O.num_threads()
    probe = min(wl.N, max(cores, 16))
    t = oracle_move_seconds(O, prob, wl, th.copy(), us.copy(), Sig, Lc, probe, 1)
    count = int(min(wl.N, max(probe, probe * seconds / max(t, 1e-3))))
    per_move = count * wl.m * (wl.L + 1)
    reps, t = 0, 0.0
    while t < seconds and reps < 1000:  # whole moves of `count` particles until ~`seconds` of work
        t += oracle_move_seconds(O, prob, wl, th.copy(), us.copy(), Sig, Lc, count, 2 + reps)
        reps += 1
    return {"value": per_move * reps / t, "unit": "grad-evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} Algorithm-1 move(s) (u block update + HMC, L={wl.L}) of {count} of "
                      f"the {wl.N} particles, FP64 C oracle with OpenMP over particles, {t:.1f} s"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from smc_workloads import logistic_1e6
    wl = logistic_1e6("bf16", n=args.n)
    O, prob, th, us, Sig, Lc = oracle_setup(wl)
    cores = O.num_threads()
    per_step_budget = max(1.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    probe = max(cores, 16)
    t = oracle_move_seconds(O, prob, wl, th.copy(), us.copy(), Sig, Lc, probe, 1)
    count = int(min(wl.N, max(probe, probe * per_step_budget / max(t, 1e-3))))
    for s in range(args.warmup):
        oracle_move_seconds(O, prob, wl, th.copy(), us.copy(), Sig, Lc, count, 2 + s)
    tot = 0.0
    for s in range(args.steps):
        tot += oracle_move_seconds(O, prob, wl, th.copy(), us.copy(), Sig, Lc, count, 100 + s)
    evals = count * wl.m * (wl.L + 1) * args.steps
    value = evals / tot
    sample = (f"per step: one Algorithm-1 move (u block update + HMC, L={wl.L}) of {count} of the "
              f"{wl.N} particles; FP64 C oracle, OpenMP over particles")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "grad-evals/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(wl, R_MOVES, 1),
           "cpu_baseline": {"value": value, "unit": "grad-evals/s", "cores": cores,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "grad-evals/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def profile_stages(args):
    """The first K stages of one run of the default workload (BF16) with the library's default
    kernel choice: k_hmc_res launches 5 (K - 1) .. 5 K - 1 are those of stage K."""
    import torch
    import paper_1805_03317_gb300 as S
    from smc_workloads import logistic_1e6
    torch.cuda.set_device(0)
    wl = logistic_1e6("bf16", n=args.n)
    X, y = device_workload(wl, torch.device("cuda", 0))
    ctx = S.smc_init(X, y, wl.family, wl.prior_mean, wl.prior_var, N=wl.N, m=wl.m, G=wl.G,
                     L=wl.L, seed=wl.seed, ess_frac=0.5, theta_bar=None,
                     hmc_kernel=args.hmc_kernel)
    a = 0.0
    for _ in range(args.profile_stages):
        a = run_stage(S, ctx, R_MOVES)
    torch.cuda.synchronize()
    print(json.dumps({"stages": args.profile_stages, "a": a}), flush=True)
    S.smc_free(ctx)


def main():
    args = parse()
    if args.profile_stages:
        profile_stages(args)
        return
    if args.gather_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(gather_leg(__import__("paper_1805_03317_gb300"), torch.device("cuda", 0),
                                    peaks()[0], tile_hint=args.gather_tile)), flush=True)
        return
    if args.batch_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(batch_leg(__import__("paper_1805_03317_gb300"), torch.device("cuda", 0))),
              flush=True)
        return
    if args.gam_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(gam_leg(__import__("paper_1805_03317_gb300"), torch.device("cuda", 0),
                                 peaks()[0], tile_hint=args.gather_tile, n=args.gam_n)), flush=True)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
