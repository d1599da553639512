"""Python front end of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module. It compiles ``smc_oracle.c`` with the host C compiler into ``oracle/_build`` and
wraps it with ctypes; the SMC driver loop below follows Algorithm 2 of the paper step by step
(reweight with an adaptive temperature, weighted moments and mass matrix, re-centring of the
control variates when asked, resample, R moves of Algorithm 1 or moves until the cloud has
decorrelated), calling the C routines for each step. Nothing here touches the CUDA library.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_margin_lock = threading.Lock()  # one margin record at a time (the C side keeps one pointer)
_lib = None

FAMILIES = {"logistic": 0, "probit": 1, "poisson": 2, "gaussian": 3, "student_t": 4}
TAG_INIT_THETA, TAG_INIT_U, TAG_UPM_BLOCK, TAG_UPM_IDX = 1, 2, 3, 4
TAG_MOMENTUM, TAG_MH_THETA, TAG_MH_U, TAG_RESAMPLE = 5, 6, 7, 8

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle (plain C99 + OpenMP) into oracle/_build/liborc.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            c_i, c_i64, c_d, c_u32, c_u64 = (ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                             ctypes.c_uint32, ctypes.c_uint64)
            L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.orc_r64.argtypes = [c_u64, c_u32, c_u32, c_u32, c_u64]
            L.orc_r64.restype = c_u64
            L.orc_index.argtypes = [c_u64, c_i64]
            L.orc_index.restype = c_i64
            L.orc_uniform.argtypes = [c_u64]
            L.orc_uniform.restype = c_d
            L.orc_normal.argtypes = [c_u64, c_u32, c_u32, c_u32, c_u64]
            L.orc_normal.restype = c_d
            L.orc_erfcx_cf.argtypes = [c_d]
            L.orc_erfcx_cf.restype = c_d
            L.orc_family.argtypes = [c_i, c_d, c_d, c_d, ctypes.POINTER(c_d),
                                     ctypes.POINTER(c_d), ctypes.POINTER(c_d)]
            L.orc_full_loglik.argtypes = [c_i, c_i64, c_i, _dp, _dp, c_d, _dp,
                                          ctypes.POINTER(c_d), ctypes.c_void_p]
            L.orc_cv_moments.argtypes = [c_i, c_i64, c_i, _dp, _dp, c_d, _dp,
                                         ctypes.POINTER(c_d), _dp, _dp]
            L.orc_log_prior.argtypes = [c_i, _dp, _dp, _dp, ctypes.c_void_p]
            L.orc_set_cv_order.argtypes = [c_i]
            L.orc_set_cv_order.restype = None
            L.orc_set_dof.argtypes = [c_d]
            L.orc_set_dof.restype = None
            L.orc_log_prior.restype = c_d
            prob = [c_i, c_i64, c_i, _dp, _dp, c_d, _dp, c_d, _dp, _dp, _dp, _dp, c_i, c_i]
            L.orc_loglik_batch.argtypes = prob + [c_i, _dp, _i64p, c_d, _dp, _dp,
                                                  ctypes.c_void_p, ctypes.c_void_p]
            L.orc_init.argtypes = [c_u64, c_i, c_i, c_i, c_i64, _dp, _dp, _dp, _i64p]
            L.orc_upm_move.argtypes = prob + [c_i, c_u64, c_u32, c_d, _dp, _i64p, _i32p]
            L.orc_hmc_move.argtypes = prob + [c_i, c_u64, c_u32, c_d, c_d, c_d, c_i, _dp, _dp,
                                              _dp, _i64p, _i32p]
            L.orc_rw_move.argtypes = prob + [c_i, c_u64, c_u32, c_d, c_d, _dp, _dp, _i64p,
                                             _i32p]
            L.orc_leapfrog.argtypes = prob + [_i64p, c_d, c_d, c_i, _dp, _dp, _dp]
            L.orc_leapfrog.restype = c_d
            L.orc_ess_at.argtypes = [c_i, _dp, _dp, _dp, c_d, c_d]
            L.orc_ess_at.restype = c_d
            L.orc_reweight.argtypes = [c_i, _dp, _dp, _dp, _dp, c_d, c_d, c_i, c_i,
                                       ctypes.POINTER(c_d), ctypes.POINTER(c_d)]
            L.orc_reweight.restype = c_d
            L.orc_cholesky.argtypes = [c_i, _dp, _dp]
            L.orc_cholesky.restype = c_i
            L.orc_moments.argtypes = [c_i, c_i, _dp, _dp, _dp, _dp, _dp]
            L.orc_moments.restype = c_i
            L.orc_resample.argtypes = [c_i, _dp, c_d, _i32p]
            L.orc_resample_multinomial.argtypes = [c_i, _dp, _dp, _i32p]
            L.orc_reweight_grid.argtypes = [c_i, _dp, _dp, _dp, _dp, c_d, c_d, c_i, c_d,
                                            ctypes.POINTER(c_d), ctypes.POINTER(c_d)]
            L.orc_reweight_grid.restype = c_d
            L.orc_num_threads.restype = c_i
            L.orc_set_margin_out.argtypes = [ctypes.c_void_p]
            L.orc_set_margin_out.restype = None
            _lib = L
    return _lib


# ----------------------------------------------------------------------------------------------
# Random numbers (same published generator and counter layout as the CUDA side, separate code)
# ----------------------------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c, k, o)
    return o


def stage_move(stage: int, move: int) -> int:
    return (stage << 8) | move


def r64(seed, tag, sm, particle, j) -> int:
    return int(lib().orc_r64(seed, tag, sm, particle, j))


def index(r, n) -> int:
    return int(lib().orc_index(r, n))


def uniform(r) -> float:
    return float(lib().orc_uniform(r))


def normal(seed, tag, sm, particle, j) -> float:
    return float(lib().orc_normal(seed, tag, sm, particle, j))


# ----------------------------------------------------------------------------------------------
# Model pieces
# ----------------------------------------------------------------------------------------------
def family(fam: str, eta: float, y: float, sigma: float = 1.0, dof: float = 5.0):
    """l, l', l'' of one row; sigma: Gaussian sd or Student-t scale, dof: Student-t nu."""
    lib().orc_set_dof(float(dof))
    l, d1, d2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_family(FAMILIES[fam], eta, y, sigma, ctypes.byref(l), ctypes.byref(d1),
                     ctypes.byref(d2))
    return l.value, d1.value, d2.value


def full_loglik(fam, X, y, theta, sigma=1.0, grad=True, dof=5.0):
    lib().orc_set_dof(float(dof))
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, p = X.shape
    ell = ctypes.c_double()
    g = np.zeros(p)
    lib().orc_full_loglik(FAMILIES[fam], n, p, X, np.ascontiguousarray(y, np.float64), sigma,
                          np.ascontiguousarray(theta, np.float64), ctypes.byref(ell),
                          g.ctypes.data if grad else None)
    return (ell.value, g) if grad else ell.value


def cv_moments(fam, X, y, theta_bar, sigma=1.0, dof=5.0):
    lib().orc_set_dof(float(dof))
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, p = X.shape
    A = ctypes.c_double()
    B = np.zeros(p)
    C = np.zeros((p, p))
    lib().orc_cv_moments(FAMILIES[fam], n, p, X, np.ascontiguousarray(y, np.float64), sigma,
                         np.ascontiguousarray(theta_bar, np.float64), ctypes.byref(A), B, C)
    return A.value, B, C


def log_prior(theta, mu, var):
    theta = np.ascontiguousarray(theta, np.float64)
    g = np.zeros(theta.shape[0])
    v = lib().orc_log_prior(theta.shape[0], theta, np.ascontiguousarray(mu, np.float64),
                            np.ascontiguousarray(var, np.float64), g.ctypes.data)
    return v, g


@dataclass
class Problem:
    """A GLM posterior: data, family, prior, control-variate centre and its moments A, B, C."""
    family: str
    X: np.ndarray            # [n, p] float64 (the stored values, upcast)
    y: np.ndarray            # [n] float64
    prior_mean: np.ndarray   # [p]
    prior_var: np.ndarray    # [p]
    sigma: float = 1.0
    theta_bar: np.ndarray | None = None
    A: float = 0.0
    B: np.ndarray | None = None
    C: np.ndarray | None = None
    cv_order: int = 2        # Taylor order of the control variates (2, or 1: first order)
    dof: float = 5.0         # Student-t degrees of freedom (sigma is then the error scale)

    def __post_init__(self):
        self.X = np.ascontiguousarray(self.X, dtype=np.float64)
        self.y = np.ascontiguousarray(self.y, dtype=np.float64)
        self.prior_mean = np.ascontiguousarray(self.prior_mean, np.float64)
        self.prior_var = np.ascontiguousarray(self.prior_var, np.float64)

    @property
    def n(self):
        return self.X.shape[0]

    @property
    def p(self):
        return self.X.shape[1]

    def set_centre(self, theta_bar):
        self.theta_bar = np.ascontiguousarray(theta_bar, np.float64)
        self.A, self.B, self.C = cv_moments(self.family, self.X, self.y, self.theta_bar,
                                            self.sigma, self.dof)

    def args(self, m, G):
        lib().orc_set_cv_order(int(self.cv_order))  # read by the estimator calls that follow
        lib().orc_set_dof(float(self.dof))
        return (FAMILIES[self.family], self.n, self.p, self.X, self.y, self.sigma,
                self.theta_bar, self.A, self.B, self.C, self.prior_mean, self.prior_var, m, G)


def newton_map(prob: Problem, iters: int = 50, tol: float = 1e-10):
    """Posterior mode (full data + prior) by Newton's method with step halving; the
    control-variate centre of the workloads (a fixed reading of Sec. 3.2's theta_bar). Where the
    negative Hessian is not positive definite (a log-density that is not concave, as the
    Student-t one far from the mode) lam I is added, lam = 1e-8 max|diag| times 10 per retry,
    which keeps the step an ascent direction (Levenberg 1944)."""
    theta = prob.prior_mean.copy()

    def damped_step(H, g):
        M = -H
        lam, scale = 0.0, max(np.max(np.abs(np.diag(M))), 1e-300)
        for _ in range(40):
            try:
                Lc = np.linalg.cholesky(M + lam * np.eye(M.shape[0]))
                return np.linalg.solve(Lc.T, np.linalg.solve(Lc, g))
            except np.linalg.LinAlgError:
                lam = 1e-8 * scale if lam == 0.0 else 10.0 * lam
        raise np.linalg.LinAlgError("no damping made the Newton matrix positive definite")

    def logpost(t):
        A, B, C = cv_moments(prob.family, prob.X, prob.y, t, prob.sigma, prob.dof)
        lp, gp = log_prior(t, prob.prior_mean, prob.prior_var)
        return A + lp, B + gp, C - np.diag(1.0 / prob.prior_var)

    f, g, H = logpost(theta)
    for _ in range(iters):
        step = damped_step(H, g)
        t = 1.0
        while True:
            cand = theta + t * step
            fc, gc, Hc = logpost(cand)
            if fc >= f or t < 1e-8:
                break
            t *= 0.5
        theta, f, g, H = cand, fc, gc, Hc
        if np.max(np.abs(t * step)) < tol:
            break
    return theta


def loglik_batch(prob: Problem, m, G, thetas, us, a=1.0, grad=True, blocks=False):
    thetas = np.ascontiguousarray(thetas, np.float64)
    us = np.ascontiguousarray(us, np.int64)
    Bn = thetas.shape[0]
    ell = np.zeros(Bn)
    s2 = np.zeros(Bn)
    g = np.zeros((Bn, prob.p)) if grad else None
    blk = np.zeros((Bn, G, 2)) if blocks else None
    lib().orc_loglik_batch(*prob.args(m, G), Bn, thetas, us, a, ell, s2,
                           g.ctypes.data if grad else None, blk.ctypes.data if blocks else None)
    out = {"ell": ell, "sigma2": s2}
    if grad:
        out["grad"] = g
    if blocks:
        out["blocks"] = blk
    return out


# ----------------------------------------------------------------------------------------------
# SMC steps (Algorithm 2) and moves (Algorithm 1)
# ----------------------------------------------------------------------------------------------
def init_particles(seed, N, p, m, n, prior_mean, prior_var):
    th = np.zeros((N, p))
    us = np.zeros((N, m), dtype=np.int64)
    lib().orc_init(seed, N, p, m, n, np.ascontiguousarray(prior_mean, np.float64),
                   np.ascontiguousarray(prior_var, np.float64), th, us)
    return th, us


class _Margins:
    """Records the MH margins (log ratio - log U per particle) of one oracle move into `out`."""

    def __init__(self, out):
        self.out = out

    def __enter__(self):
        if self.out is not None:
            L = lib()
            _margin_lock.acquire()
            L.orc_set_margin_out(self.out.ctypes.data)

    def __exit__(self, *exc):
        if self.out is not None:
            lib().orc_set_margin_out(None)
            _margin_lock.release()


def _margin_buffer(margins, N):
    if margins is None:
        return None
    if margins.dtype != np.float64 or margins.shape != (N,) or not margins.flags.c_contiguous:
        raise ValueError("margins must be a contiguous float64 array of one value per particle")
    return margins


def upm_move(prob, m, G, seed, stage, move, a, thetas, us, margins=None):
    """Block pseudo-marginal u update (Algorithm 1 step 1). margins: optional float64 [N] that
    receives log r - log U per particle (the decision's distance from the MH threshold)."""
    N = thetas.shape[0]
    acc = np.zeros(N, dtype=np.int32)
    args = prob.args(m, G)
    with _Margins(_margin_buffer(margins, N)):
        lib().orc_upm_move(*args, N, seed, stage_move(stage, move), a,
                           np.ascontiguousarray(thetas, np.float64), us, acc)
    return acc


def hmc_move(prob, m, G, seed, stage, move, a, eps, L, Sigma, Lc, thetas, us, jitter=0.3,
             margins=None):
    """HMC move of theta given u (Algorithm 1 step 2); jitter > 0: each particle's step size is
    uniform on eps [1 - jitter, 1 + jitter]. margins: optional float64 [N] that receives
    H0 - H1 - log U per particle."""
    N = thetas.shape[0]
    acc = np.zeros(N, dtype=np.int32)
    args = prob.args(m, G)
    with _Margins(_margin_buffer(margins, N)):
        lib().orc_hmc_move(*args, N, seed, stage_move(stage, move), a, eps, jitter, L,
                           np.ascontiguousarray(Sigma, np.float64),
                           np.ascontiguousarray(Lc, np.float64), thetas,
                           np.ascontiguousarray(us, np.int64), acc)
    return acc


def leapfrog(prob, m, G, u, a, eps, L, Sigma, theta, rho):
    """One leapfrog trajectory of the HMC move (the same routine the move runs) from (theta, rho)
    at fixed u: returns (theta_L, rho_L, log target at theta_L). Test support."""
    th = np.array(theta, dtype=np.float64)
    r = np.array(rho, dtype=np.float64)
    lt = lib().orc_leapfrog(*prob.args(m, G), np.ascontiguousarray(u, np.int64), a, eps, L,
                            np.ascontiguousarray(Sigma, np.float64), th, r)
    return th, r, lt


def rw_move(prob, m, G, seed, stage, move, a, eps, Lc, thetas, us):
    """Random-walk Metropolis move of theta given u, proposal N(theta, eps^2 Lc Lc')."""
    N = thetas.shape[0]
    acc = np.zeros(N, dtype=np.int32)
    lib().orc_rw_move(*prob.args(m, G), N, seed, stage_move(stage, move), a, eps,
                      np.ascontiguousarray(Lc, np.float64), thetas,
                      np.ascontiguousarray(us, np.int64), acc)
    return acc


def ess_at(logW, ell, sig2, a, D):
    return float(lib().orc_ess_at(len(logW), np.ascontiguousarray(logW, np.float64),
                                  np.ascontiguousarray(ell, np.float64),
                                  np.ascontiguousarray(sig2, np.float64), a, D))


def reweight(logW, ell, sig2, a, tau, K=16, rounds=10):
    """Returns (a_new, logW_new, W_new, log_z_inc, ess); inputs are not modified."""
    lw = np.array(logW, dtype=np.float64)
    W = np.zeros_like(lw)
    lz = ctypes.c_double()
    ess = ctypes.c_double()
    a_new = lib().orc_reweight(len(lw), lw, W, np.ascontiguousarray(ell, np.float64),
                               np.ascontiguousarray(sig2, np.float64), a, tau, K, rounds,
                               ctypes.byref(lz), ctypes.byref(ess))
    return float(a_new), lw, W, lz.value, ess.value


def reweight_grid(logW, ell, sig2, a, tau, S=1024, decades=16.0):
    """The paper's grid rule (Sec. 2.3) on S geometric increments; same returns as reweight."""
    lw = np.array(logW, dtype=np.float64)
    W = np.zeros_like(lw)
    lz = ctypes.c_double()
    ess = ctypes.c_double()
    a_new = lib().orc_reweight_grid(len(lw), lw, W, np.ascontiguousarray(ell, np.float64),
                                    np.ascontiguousarray(sig2, np.float64), a, tau, S, decades,
                                    ctypes.byref(lz), ctypes.byref(ess))
    return float(a_new), lw, W, lz.value, ess.value


def cholesky(S):
    S = np.ascontiguousarray(S, np.float64)
    Lc = np.zeros_like(S)
    rc = lib().orc_cholesky(S.shape[0], S, Lc)
    return Lc if rc == 0 else None


def moments(W, thetas):
    N, p = thetas.shape
    mean = np.zeros(p)
    S = np.zeros((p, p))
    Lc = np.zeros((p, p))
    rc = lib().orc_moments(N, p, np.ascontiguousarray(W, np.float64),
                           np.ascontiguousarray(thetas, np.float64), mean, S, Lc)
    return mean, S, Lc, rc


def resample(W, U):
    W = np.ascontiguousarray(W, np.float64)
    anc = np.zeros(W.shape[0], dtype=np.int32)
    lib().orc_resample(W.shape[0], W, U, anc)
    return anc


def resample_multinomial(W, U):
    """Multinomial resampling (Sec. 2.2): U[i] is offspring i's uniform."""
    W = np.ascontiguousarray(W, np.float64)
    anc = np.zeros(W.shape[0], dtype=np.int32)
    lib().orc_resample_multinomial(W.shape[0], W, np.ascontiguousarray(U, np.float64), anc)
    return anc


def multinomial_uniforms(seed, stage, N):
    """Offspring i's uniform: the second 64-bit draw of its block in the stage's resampling
    stream (the first draw of offspring 0 is the systematic scheme's U)."""
    return np.array([uniform(r64(seed, TAG_RESAMPLE, stage_move(stage, 0), i, 1))
                     for i in range(N)])


def num_threads() -> int:
    return int(lib().orc_num_threads())


@dataclass
class SMCConfig:
    N: int
    m: int
    G: int
    L: int
    R: int
    seed: int
    tau: float = 0.5
    K: int = 16
    rounds: int = 10
    eps0: float | None = None      # default 0.5 * p^(-1/4)
    max_stages: int = 1000
    recentre: int = 0              # 1: Algorithm 2 (d), theta_bar = the reweighted particle mean
                                   # after the reweighting; 2: the weighted mean of the current
                                   # cloud at the start of the stage, estimates refreshed before
                                   # the reweighting
    resampling: str = "systematic"  # or "multinomial" (the paper's scheme)
    grid_points: int = 0           # > 0: the paper's grid rule for the temperature (Sec. 2.3)
    grid_decades: float = 16.0
    adaptive: tuple | None = None  # (R_max, rho_max, quantile): moves until decorrelated
    theta_move: str = "hmc"        # or "rw": random-walk Metropolis (Sec. 4.2's comparison)
    eps_jitter: float = 0.3        # HMC: per-particle step size uniform on eps [1 -+ jitter]


@dataclass
class SMCState:
    stage: int
    a: float
    eps: float
    thetas: np.ndarray
    us: np.ndarray
    logW: np.ndarray
    W: np.ndarray
    ell: np.ndarray
    sig2: np.ndarray
    log_z: float = 0.0
    Sigma: np.ndarray | None = None   # mass-matrix inverse of the last stage (prior covariance at first)
    Lc: np.ndarray | None = None
    history: list = field(default_factory=list)


def componentwise_correlation(th0, th):
    """Correlation across particles of each component between two clouds (a component with no
    spread in either cloud counts as 1)."""
    d0 = th0 - th0.mean(axis=0)
    d1 = th - th.mean(axis=0)
    xx, yy, xy = (d0 * d0).sum(axis=0), (d1 * d1).sum(axis=0), (d0 * d1).sum(axis=0)
    ok = (xx > 0) & (yy > 0)
    return np.where(ok, xy / np.sqrt(np.where(ok, xx * yy, 1.0)), 1.0)


def decorrelated(th0, th, rho_max, quantile):
    """The adaptive-R rule (Sec. 3.4, after Buchholz et al.): the ceil(quantile p)-th smallest
    componentwise correlation between the starting and the current cloud is at most rho_max."""
    rho = np.sort(componentwise_correlation(th0, th))
    p = rho.shape[0]
    k = min(max(math.ceil(quantile * p) - 1, 0), p - 1)
    return bool(rho[k] <= rho_max)


def smc_init(prob: Problem, cfg: SMCConfig) -> SMCState:
    """Algorithm 2 step 1: particles from the prior and p(u), equal weights, cached estimates."""
    th, us = init_particles(cfg.seed, cfg.N, prob.p, cfg.m, prob.n, prob.prior_mean,
                            prob.prior_var)
    out = loglik_batch(prob, cfg.m, cfg.G, th, us, a=0.0, grad=False)
    eps = cfg.eps0 if cfg.eps0 is not None else 0.5 * prob.p ** -0.25
    logW = np.full(cfg.N, -math.log(cfg.N))
    Sigma0 = np.diag(prob.prior_var)
    return SMCState(0, 0.0, eps, th, us, logW, np.exp(logW), out["ell"], out["sigma2"],
                    Sigma=Sigma0, Lc=np.linalg.cholesky(Sigma0))


def smc_stage(prob: Problem, cfg: SMCConfig, st: SMCState):
    """One pass of Algorithm 2's loop body: (a) stage+1, (b)-(c) temperature and reweighting,
    (d) weighted moments and mass matrix, (e) resampling, (f) R moves of Algorithm 1."""
    st.stage += 1
    s = st.stage
    if cfg.recentre == 2:  # centre at the current cloud; the cache follows the new estimator
        mean0, _, _, _ = moments(st.W, st.thetas)
        prob.set_centre(mean0)
        out = loglik_batch(prob, cfg.m, cfg.G, st.thetas, st.us, a=st.a, grad=False)
        st.ell, st.sig2 = out["ell"], out["sigma2"]
    if cfg.grid_points > 0:
        a_new, logW, W, lz, ess = reweight_grid(st.logW, st.ell, st.sig2, st.a, cfg.tau,
                                                cfg.grid_points, cfg.grid_decades)
    else:
        a_new, logW, W, lz, ess = reweight(st.logW, st.ell, st.sig2, st.a, cfg.tau, cfg.K,
                                           cfg.rounds)
    mean, Sigma, Lc, rc = moments(W, st.thetas)
    if rc >= 0:  # a covariance that is not positive definite (e.g. N = 1) keeps the previous one
        st.Sigma, st.Lc = Sigma, Lc
    if cfg.recentre == 1:  # new control variates at the weighted mean: A, B, C once per stage
        prob.set_centre(mean)
    if cfg.resampling == "multinomial":
        anc = resample_multinomial(W, multinomial_uniforms(cfg.seed, s, cfg.N))
    else:
        anc = resample(W, uniform(r64(cfg.seed, TAG_RESAMPLE, stage_move(s, 0), 0, 0)))
    st.thetas = st.thetas[anc].copy()
    st.us = st.us[anc].copy()
    st.a = a_new
    st.log_z += lz
    st.logW = np.full(cfg.N, -math.log(cfg.N))
    st.W = np.exp(st.logW)
    acc_u = acc_t = 0
    R_max = cfg.R if cfg.adaptive is None else int(cfg.adaptive[0])
    th0 = st.thetas.copy()
    R = 0
    while R < R_max:
        acc_u += int(upm_move(prob, cfg.m, cfg.G, cfg.seed, s, R, st.a, st.thetas, st.us).sum())
        if cfg.theta_move == "rw":
            acc_t += int(rw_move(prob, cfg.m, cfg.G, cfg.seed, s, R, st.a, st.eps, st.Lc,
                                 st.thetas, st.us).sum())
        else:
            acc_t += int(hmc_move(prob, cfg.m, cfg.G, cfg.seed, s, R, st.a, st.eps, cfg.L,
                                  st.Sigma, st.Lc, st.thetas, st.us, cfg.eps_jitter).sum())
        R += 1
        if cfg.adaptive is not None:
            _, rho_max, q = cfg.adaptive
            if decorrelated(th0, st.thetas, rho_max, q):
                break
    out = loglik_batch(prob, cfg.m, cfg.G, st.thetas, st.us, a=st.a, grad=False)
    st.ell, st.sig2 = out["ell"], out["sigma2"]
    rate = acc_t / float(cfg.N * R)
    st.history.append(dict(stage=s, a=st.a, ess=ess, log_z_inc=lz, eps=st.eps,
                           acc_u=acc_u / float(cfg.N * R), acc_theta=rate, R=R))
    target = 0.234 if cfg.theta_move == "rw" else 0.65  # acceptance the step size is steered to
    st.eps = st.eps * min(2.0, max(0.5, math.exp(rate - target)))
    return st


def smc_run(prob: Problem, cfg: SMCConfig) -> SMCState:
    st = smc_init(prob, cfg)
    while st.a < 1.0 and st.stage < cfg.max_stages:
        smc_stage(prob, cfg, st)
    return st
