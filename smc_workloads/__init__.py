"""Seeded synthetic inputs shaped like the paper's GLM workloads.

This module only generates data (covariates, responses, priors and run settings). It holds none
of the method's arithmetic and is the one piece shared by the CUDA tests, the oracle tests and the
benchmark. Every array is produced from ``numpy.random.Generator(PCG64(seed))``.

Stored precision: ``x_dtype`` names how X is stored on the device ("f64", "f32" or "bf16").
``Workload.X`` always holds the *stored* values upcast to float64, so the oracle sees exactly what
the GPU reads; ``Workload.X_store`` holds the raw storage (float64, float32, or the uint16 bit
patterns of bfloat16). The response y is stored as float64 for "f64" problems and float32
otherwise; ``Workload.y`` is its float64 upcast.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 20180508


def round_to_bf16_bits(a32: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); returns the uint16 bits."""
    b = np.ascontiguousarray(a32, dtype=np.float32).view(np.uint32)
    b = (b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) >> np.uint32(16)
    return b.astype(np.uint16)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@dataclass
class Workload:
    name: str
    family: str
    x_dtype: str
    X: np.ndarray          # [n, p] float64: stored values, upcast
    X_store: np.ndarray    # [n, p] raw storage
    y: np.ndarray          # [n] float64: stored values, upcast
    y_store: np.ndarray    # [n] raw storage (float64 or float32)
    prior_mean: np.ndarray
    prior_var: np.ndarray
    N: int
    m: int
    G: int
    L: int
    R: int
    seed: int
    sigma: float = 1.0
    theta_true: np.ndarray | None = None
    dof: float = 5.0       # Student-t degrees of freedom (sigma is then the error scale)

    @property
    def n(self) -> int:
        return self.X_store.shape[0]

    @property
    def p(self) -> int:
        return self.X_store.shape[1]


def _store(X: np.ndarray, y: np.ndarray, x_dtype: str, upcast: bool = True):
    if x_dtype == "f64":
        Xs = np.ascontiguousarray(X, dtype=np.float64)
        ys = np.ascontiguousarray(y, dtype=np.float64)
        return Xs, Xs, ys, ys
    ys = np.ascontiguousarray(y, dtype=np.float32)
    if x_dtype == "f32":
        Xs = np.ascontiguousarray(X, dtype=np.float32)
        return Xs.astype(np.float64), Xs, ys.astype(np.float64), ys
    if x_dtype == "bf16":
        bits = round_to_bf16_bits(np.asarray(X, dtype=np.float32))
        return (bf16_bits_to_f64(bits) if upcast else None), bits, ys.astype(np.float64), ys
    raise ValueError(x_dtype)


def _respond(rng, family: str, eta: np.ndarray, sigma: float = 1.0, dof: float = 5.0) -> np.ndarray:
    if family == "logistic":
        return (rng.random(eta.shape[0]) < 1.0 / (1.0 + np.exp(-eta))).astype(np.float64)
    if family == "probit":
        from scipy.special import ndtr
        return (rng.random(eta.shape[0]) < ndtr(eta)).astype(np.float64)
    if family == "poisson":
        return rng.poisson(np.exp(eta)).astype(np.float64)
    if family == "gaussian":
        return eta + sigma * rng.standard_normal(eta.shape[0])
    if family == "student_t":
        return eta + sigma * rng.standard_t(dof, size=eta.shape[0])
    raise ValueError(family)


def small_glm(family: str = "logistic", n: int = 2000, p: int = 5, N: int = 64, m: int = 50,
              G: int = 5, L: int = 5, R: int = 2, x_dtype: str = "f64", seed: int = 1,
              sigma: float = 0.5, theta_scale: float = 0.5, prior_var: float = 10.0,
              x_scale: float = 1.0, dof: float = 5.0) -> Workload:
    """Small seeded GLM (intercept + iid N(0, x_scale^2) covariates) for parity and pin tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.empty((n, p))
    X[:, 0] = 1.0
    X[:, 1:] = x_scale * rng.standard_normal((n, p - 1))
    theta = theta_scale * rng.standard_normal(p)
    Xs64, Xs, _, _ = _store(X, np.zeros(n), x_dtype)
    y = _respond(rng, family, Xs64 @ theta, sigma, dof)
    Xd, Xs, yd, ys = _store(X, y, x_dtype)
    return Workload(f"small-{family}", family, x_dtype, Xd, Xs, yd, ys, np.zeros(p),
                    np.full(p, prior_var), N, m, G, L, R, seed, sigma, theta, dof)


def logistic_1e4(seed_offset: int = 0) -> Workload:
    """Plain method in FP64: logistic regression, n=10,000, p=5 (intercept + 4 iid N(0,1)),
    theta_true ~ N(0, 0.5^2 I), prior N(0, 10 I); N=256 particles, m=100, G=10, L=10, R=5."""
    seed = BASE_SEED + 0 + seed_offset
    rng = np.random.Generator(np.random.PCG64(seed))
    n, p = 10_000, 5
    X = np.empty((n, p))
    X[:, 0] = 1.0
    X[:, 1:] = rng.standard_normal((n, p - 1))
    theta = 0.5 * rng.standard_normal(p)
    y = _respond(rng, "logistic", X @ theta)
    Xd, Xs, yd, ys = _store(X, y, "f64")
    return Workload("logistic-n1e4-p5-f64", "logistic", "f64", Xd, Xs, yd, ys, np.zeros(p),
                    np.full(p, 10.0), 256, 100, 10, 10, 5, seed, 1.0, theta)


def logistic_1e6(x_dtype: str = "bf16", n: int = 1_000_000) -> Workload:
    """Logistic regression at scale: n=1,000,000, p=20 (intercept + 19 N(0,1) covariates with
    AR(1) correlation 0.5 across columns), theta_true ~ N(0, 0.3^2 I), prior N(0, 10 I);
    N=4096 particles, m=1000, G=10, L=20, R=5. X stored as FP32 or BF16."""
    seed = BASE_SEED + 1
    rng = np.random.Generator(np.random.PCG64(seed))
    p, rho = 20, 0.5
    X = np.empty((n, p), dtype=np.float32)
    X[:, 0] = 1.0
    prev = rng.standard_normal(n)
    X[:, 1] = prev
    s = math.sqrt(1.0 - rho * rho)
    for c in range(2, p):
        prev = rho * prev + s * rng.standard_normal(n)
        X[:, c] = prev
    theta = 0.3 * rng.standard_normal(p)
    Xs64, _, _, _ = _store(X, np.zeros(n), x_dtype)
    y = _respond(rng, "logistic", Xs64 @ theta)
    Xd, Xs, yd, ys = _store(X, y, x_dtype)
    return Workload(f"logistic-n1e6-p20-{x_dtype}", "logistic", x_dtype, Xd, Xs, yd, ys,
                    np.zeros(p), np.full(p, 10.0), 4096, 1000, 10, 20, 5, seed, 1.0, theta)


def student_t_5e5(x_dtype: str = "bf16", n: int = 500_000, N: int = 4096, L: int = 20) -> Workload:
    """Student-t regression of the paper's Experiment 2 (Sec. 4.3) in shape: n=500,000, p=50
    covariates with unit variances and pairwise correlation 0.9 (x = sqrt(0.9) z0 + sqrt(0.1) z_j),
    theta_true ~ U(-5, 5), errors t_5 with unit scale, prior N(0, 10 I); m = 1250 (sample
    fraction 0.0025), G = 100, R = 5. X stored as BF16 (or FP32)."""
    seed = BASE_SEED + 5
    rng = np.random.Generator(np.random.PCG64(seed))
    p = 50
    z0 = rng.standard_normal(n)
    X = (math.sqrt(0.9) * z0[:, None] + math.sqrt(0.1) * rng.standard_normal((n, p))).astype(
        np.float32)
    theta = rng.uniform(-5.0, 5.0, p)
    Xs64, _, _, _ = _store(X, np.zeros(n), x_dtype)
    y = _respond(rng, "student_t", Xs64 @ theta, 1.0, 5.0)
    Xd, Xs, yd, ys = _store(X, y, x_dtype)
    return Workload(f"student-t-n5e5-p50-{x_dtype}", "student_t", x_dtype, Xd, Xs, yd, ys,
                    np.zeros(p), np.full(p, 10.0), N, 1250, 100, L, 5, seed, 1.0, theta, 5.0)


def poisson_5e6(x_dtype: str = "bf16", n: int = 5_000_000, upcast: bool = True) -> Workload:
    """Poisson regression: n=5,000,000, p=50 (intercept + 49 N(0, 0.1^2) covariates),
    theta_true ~ N(0, 0.2^2 I) with intercept 1.0, prior N(0, 0.1 I); N=8192, m=2000, G=20,
    L=20, R=5. X stored as BF16. upcast=False skips the float64 copy of X (Workload.X is None)."""
    seed = BASE_SEED + 2
    rng = np.random.Generator(np.random.PCG64(seed))
    p = 50
    X = np.empty((n, p), dtype=np.float32)
    X[:, 0] = 1.0
    X[:, 1:] = 0.1 * rng.standard_normal((n, p - 1), dtype=np.float32)
    theta = 0.2 * rng.standard_normal(p)
    theta[0] = 1.0
    _, Xs, _, _ = _store(X, np.zeros(n), x_dtype, upcast=False)
    Xv = bf16_bits_to_f64(Xs).astype(np.float32) if x_dtype == "bf16" else Xs
    y = _respond(rng, "poisson", Xv.astype(np.float64) @ theta)
    del Xv
    Xd, Xs, yd, ys = _store(X, y, x_dtype, upcast=upcast)
    return Workload(f"poisson-n5e6-p50-{x_dtype}", "poisson", x_dtype, Xd, Xs, yd, ys,
                    np.zeros(p), np.full(p, 0.1), 8192, 2000, 20, 20, 5, seed, 1.0, theta)


GAM_KNOTS = np.r_[[0.0] * 4, np.arange(1, 7) / 7.0, [1.0] * 4]  # clamped cubic, 6 interior knots


def gam_basis(u: np.ndarray) -> np.ndarray:
    """Cubic B-spline basis (10 functions, 6 equally spaced interior knots on [0, 1], clamped ends)
    of every column of u [n, q] in [0, 1): returns [n, 10 q] float32, covariate-major. Only the
    four functions that are nonzero on a point's knot span are evaluated (de Boor's triangular
    recurrence for the basis functions of one span)."""
    n, q = u.shape
    out = np.zeros((n, 10 * q), dtype=np.float32)
    flat = out.reshape(-1)
    t = GAM_KNOTS.astype(np.float32)
    base = np.arange(n, dtype=np.int64) * (10 * q)
    for j in range(q):
        x = u[:, j].astype(np.float32)
        span = np.minimum((x * 7).astype(np.int64), 6)
        mu = 3 + span  # t[mu] <= x < t[mu + 1]
        N = [np.ones(n, dtype=np.float32)]
        left = [None] * 4
        right = [None] * 4
        for d in range(1, 4):
            left[d] = x - t[mu + 1 - d]
            right[d] = t[mu + d] - x
            saved = np.zeros(n, dtype=np.float32)
            nxt = []
            for r in range(d):
                tmp = N[r] / (right[r + 1] + left[d - r])
                nxt.append(saved + right[r + 1] * tmp)
                saved = left[d - r] * tmp
            nxt.append(saved)
            N = nxt
        idx = base + 10 * j + span
        for r in range(4):
            flat[idx + r] = N[r]
    return out


def gam_1e7(x_dtype: str = "bf16", n: int = 10_000_000, N: int = 16384, m: int = 5000,
            upcast: bool = True, chunk: int = 1_000_000) -> Workload:
    """Generalized additive model, Gaussian response with known sigma = 0.5: 10 covariates
    iid U[0, 1), each expanded into 10 cubic B-spline functions, plus an intercept (p = 101).
    True smooth functions: covariate j has a * sin(2 pi b x + c) (even j) or a * (x - c)^2 (odd j)
    with a, b, c drawn from the seed; intercept 1. Prior N(0, 100 I). N=16384, m=5000, G=10,
    L=25, R=5. Rows are generated in chunks (the random stream depends on the chunk size)."""
    seed = BASE_SEED + 4
    rng = np.random.Generator(np.random.PCG64(seed))
    q, p = 10, 101
    amp = rng.uniform(0.5, 2.0, q)
    freq = rng.uniform(0.5, 2.0, q)
    shift = rng.uniform(0.0, 1.0, q)
    sigma = 0.5
    Xs = np.empty((n, p), dtype=np.uint16 if x_dtype == "bf16" else
                  (np.float32 if x_dtype == "f32" else np.float64))
    y = np.empty(n)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        u = rng.random((r1 - r0, q))
        f = np.ones(r1 - r0)
        for j in range(q):
            if j % 2 == 0:
                f += amp[j] * np.sin(2 * np.pi * freq[j] * u[:, j] + 2 * np.pi * shift[j])
            else:
                f += amp[j] * (u[:, j] - shift[j]) ** 2
        y[r0:r1] = f + sigma * rng.standard_normal(r1 - r0)
        B = np.empty((r1 - r0, p), dtype=np.float32)
        B[:, 0] = 1.0
        B[:, 1:] = gam_basis(u)
        if x_dtype == "bf16":
            Xs[r0:r1] = round_to_bf16_bits(B)
        else:
            Xs[r0:r1] = B
    ys = y.astype(np.float64 if x_dtype == "f64" else np.float32)
    if x_dtype == "bf16":
        Xd = bf16_bits_to_f64(Xs) if upcast else None
    else:
        Xd = Xs.astype(np.float64) if upcast else None
    return Workload(f"gam-n{n}-p101-{x_dtype}", "gaussian", x_dtype, Xd, Xs, ys.astype(np.float64),
                    ys, np.zeros(p), np.full(p, 100.0), N, m, 10, 25, 5, seed, sigma, None)


def batch_uneven(P: int = 64, N: int = 1024, G: int = 10, L: int = 20, R: int = 5,
                 n_lo: float = 1e4, n_hi: float = 1e6, seed_offset: int = 0,
                 upcast: bool = True) -> list:
    """Batched uneven posteriors: P independent regressions, half logistic and half probit, n
    log-uniform in [n_lo, n_hi], p uniform in {5, ..., 40} (intercept + N(0, 1) covariates),
    theta_true ~ N(0, 0.3^2 I), prior N(0, 10 I); N particles each, m = ceil(0.001 n) clamped to
    [100, 1000], G blocks, L leapfrog steps, R moves. X stored in BF16. Each problem has its own
    seed (BASE_SEED + 3, then a per-problem stream). upcast=False leaves Workload.X as None."""
    seed = BASE_SEED + 3 + seed_offset
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(P):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        p = int(rng.integers(5, 41))
        fam = "logistic" if q % 2 == 0 else "probit"
        m = int(min(1000, max(100, math.ceil(0.001 * n))))
        prng = np.random.Generator(np.random.PCG64([seed, q]))
        X = np.empty((n, p), dtype=np.float32)
        X[:, 0] = 1.0
        X[:, 1:] = prng.standard_normal((n, p - 1), dtype=np.float32)
        theta = 0.3 * prng.standard_normal(p)
        bits = round_to_bf16_bits(X)
        del X
        Xd = bf16_bits_to_f64(bits)
        y = _respond(prng, fam, Xd @ theta)
        if not upcast:
            Xd = None
        ys = y.astype(np.float32)
        out.append(Workload(f"batch{q}-{fam}-n{n}-p{p}", fam, "bf16", Xd, bits, ys.astype(np.float64),
                            ys, np.zeros(p), np.full(p, 10.0), N, m, G, L, R, seed * 1000 + q, 1.0,
                            theta))
    return out
