"""GPU parity at the workloads' own shapes, through the C ABI, against the FP64 oracle.

- The resident HMC trajectory kernel at the headline shape: logistic regression with the AR(1)
  covariate design of the n = 10^6 workload (at n = 2*10^5 here), p = 20, m = 1000, G = 10,
  L = 20, the 20-slot tile, BF16 and FP32 storage; one Algorithm-1 move from prior draws (rows
  far from the centre: the exp/log form of the logistic increment), from a mid spread (both
  forms in one warp) and at a late-stage spread (the cumulant series).
- The logistic per-row increment and its derivative on every branch, row by row.
- The streamed estimator's sigma2_hat at prior draws of the same shape, particle by particle.
- The plain FP64 workload (n = 10^4, p = 5, N = 256, m = 100, G = 10, L = 10, R = 5) run to a = 1
  over ten seeds against an importance-sampling log marginal likelihood and posterior mean.
- The Poisson workload at full size (n = 5*10^6, p = 50, BF16, N = 8192, m = 2000, G = 20): the
  gradient of the annealed target at 32 random particles of every stage against central
  differences of the oracle's FP64 estimator.

MH decisions are compared where the oracle's decision margin (log ratio - log U) exceeds the
rounding of the reduced-precision side; every other particle must agree."""
import math

import numpy as np
import pytest
import torch

from gpu_common import ell_scale, make_pair, state_round
from oracle import oracle as O

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
HMC_20_SLOT = 8  # hmc_kernel value of the resident 20-slot, 4-warp tile (both storage types)
HMC_TC = 10      # the tensor-core trajectory kernel (BF16 storage)


def S():
    import paper_1805_03317_gb300 as pkg
    return pkg


def _headline(x_dtype, N=256):
    from smc_workloads import logistic_1e6
    wl = logistic_1e6(x_dtype, n=200_000)
    wl.N = N
    return wl


# regime: (cloud, temperature before the reweighting, leapfrog step)
REGIMES = {"prior": ("prior", 0.0, 0.4), "mid": (0.08, 0.002, 0.3), "late": (0.01, 0.6, 0.2)}


@pytest.mark.parametrize("kernel,x_dtype", [(HMC_20_SLOT, "bf16"), (HMC_20_SLOT, "f32"),
                                            (HMC_TC, "bf16")])
@pytest.mark.parametrize("regime", ["prior", "mid", "late"])
def test_resident_trajectory_at_the_headline_shape(kernel, x_dtype, regime):
    """One move of the resident trajectory kernels (the 20-slot CUDA-core tile and the tensor-core
    kernel) against the oracle's move on the same cloud."""
    wl = _headline(x_dtype)
    prob, ctx = make_pair(wl, hmc_kernel=kernel)
    cloud, a0, eps = REGIMES[regime]
    rng = np.random.default_rng(17)
    if cloud == "prior":
        th, _ = O.init_particles(99, wl.N, wl.p, wl.m, wl.n, wl.prior_mean, wl.prior_var)
    else:
        th = prob.theta_bar + cloud * rng.standard_normal((wl.N, wl.p))
    th = state_round(th, x_dtype)
    u = rng.integers(0, wl.n, size=(wl.N, wl.m)).astype(np.int64)
    W = np.full(wl.N, 1.0 / wl.N)
    S().smc_set_particles(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV),
                          torch.from_numpy(W).to(DEV))
    S().smc_set_scalars(ctx, 2, a0, eps, 0.0)
    a, _, _ = S().smc_reweight(ctx)  # stage 3; the mass matrix comes from this cloud
    S().smc_move(ctx, 1)
    th_g, u_g, _ = S().smc_get_particles(ctx)
    th_g, u_g = th_g.cpu().double().numpy(), u_g.cpu().numpy()
    ell_g, s2_g, blk_g = (t.cpu().numpy() for t in S().smc_get_cache(ctx))
    S().smc_free(ctx)

    ref = O.loglik_batch(prob, wl.m, wl.G, th, u, grad=False)
    ra, _, rW, _, _ = O.reweight(np.log(W), ref["ell"], ref["sigma2"], a0, 0.5)
    assert a == pytest.approx(ra, rel=1e-5, abs=1e-12)
    _, Sig, Lc, _ = O.moments(rW, th)
    th_o, u_o = th.copy(), u.copy()
    mu = np.zeros(wl.N)
    mh = np.zeros(wl.N)
    O.upm_move(prob, wl.m, wl.G, wl.seed, 3, 0, ra, th_o, u_o, margins=mu)
    O.hmc_move(prob, wl.m, wl.G, wl.seed, 3, 0, ra, eps, wl.L, Sig, Lc, th_o, u_o, margins=mh)

    # u update: identical indices wherever the decision is not within rounding of the threshold
    clear_u = np.abs(mu) > 1e-3
    assert clear_u.mean() >= 0.95
    assert np.array_equal(u_g[clear_u], u_o[clear_u])
    same_u = np.all(u_g == u_o, axis=1)
    # theta move: same decision wherever the oracle's margin is clear of FP32 rounding
    clear = clear_u & same_u & (np.abs(mh) > 1e-2)
    assert clear.mean() >= 0.9
    moved_g = np.any(th_g != th, axis=1)
    moved_o = mh > 0
    assert np.array_equal(moved_g[clear], moved_o[clear])
    both = clear & moved_o
    assert both.sum() >= 25, both.sum()
    # end points within 2e-4 of the particle's own size: FP32 leapfrog rounding grows with the
    # distance travelled, which is several units from prior draws
    th_scale = np.maximum(np.max(np.abs(th_o[both]), axis=1, keepdims=True), 0.1)
    assert np.max(np.abs(th_g[both] - th_o[both]) / th_scale) <= 2e-4

    # the cache after the move: the resident kernel's end point (accepted) or the u update's
    # estimates (rejected), against the oracle at the oracle's end state
    ref2 = O.loglik_batch(prob, wl.m, wl.G, th_o, u_o, grad=False, blocks=True)
    scale = ell_scale(prob, th_o, ref2["ell"])
    ok = clear
    assert np.all(np.abs(ell_g[ok] - ref2["ell"][ok]) <= 1e-5 * scale[ok])
    s2o = ref2["sigma2"]
    assert np.all(np.abs(s2_g[ok] - s2o[ok]) <= 1e-4 * np.abs(s2o[ok]) + 1e-9 * scale[ok])
    # block sums (sum d, sum d^2 per block of u) to 1e-4 of the largest, the bar the cache tests use
    bo = ref2["blocks"]
    assert np.max(np.abs(blk_g - bo)[ok]) <= 1e-4 * np.max(np.abs(bo[ok]))
    if regime == "prior":
        # far from the centre: the rows' increments share a large mean, so the one-pass variance
        # would cancel; sigma2_hat is still held to 1e-4 of itself
        assert np.median(s2o[ok]) > 1e6


@pytest.mark.parametrize("x_dtype", ["bf16", "f32"])
def test_streamed_estimator_sigma2_far_from_the_centre(x_dtype):
    """loglik_grad on prior draws at the headline shape (the streamed kernel): sigma2_hat within 1e-4
    of the oracle's, particle by particle, l_hat and the gradient within the workloads' bars."""
    wl = _headline(x_dtype)
    prob, ctx = make_pair(wl)
    th, u = O.init_particles(5, wl.N, wl.p, wl.m, wl.n, wl.prior_mean, wl.prior_var)
    th = state_round(th, x_dtype)
    a = 1e-4
    g, ell, s2 = S().loglik_grad(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV), a)
    S().smc_free(ctx)
    ref = O.loglik_batch(prob, wl.m, wl.G, th, u, a=a)
    scale = ell_scale(prob, th, ref["ell"])
    assert np.all(np.abs(ell.cpu().numpy() - ref["ell"]) <= 1e-5 * scale)
    s2o = ref["sigma2"]
    assert np.median(s2o) > 1e6
    assert np.all(np.abs(s2.cpu().numpy() - s2o) <= 1e-4 * np.abs(s2o))
    gs = np.maximum(np.max(np.abs(ref["grad"]), axis=1, keepdims=True), 1.0)
    assert np.max(np.abs(g.cpu().double().numpy() - ref["grad"]) / gs) <= 1e-4


_IS_CACHE = {}


def _importance_reference(wl):
    from logml_reference import importance_reference
    if "ref" not in _IS_CACHE:
        _IS_CACHE["ref"] = importance_reference(wl.X, wl.y, wl.prior_var)
    return _IS_CACHE["ref"]


def _plain_run(wl, seed, N):
    from gpu_common import device_arrays
    X, y = device_arrays(wl)
    ctx = S().smc_init(X, y, "logistic", wl.prior_mean, wl.prior_var, N=N, m=wl.m, G=wl.G,
                       L=wl.L, seed=seed, ess_frac=0.5, theta_bar=None)
    runner = S().SubsampledSMC.__new__(S().SubsampledSMC)
    runner.ctx, runner.history = ctx, []
    st = runner.run(wl.R)
    th, _, W = S().smc_get_particles(ctx)
    mean = (th.double() * W[:, None]).sum(0).cpu().numpy()
    S().smc_free(ctx)
    return st["log_z"], mean


@pytest.mark.parametrize("N", [256, 2048])
def test_plain_fp64_workload_recovers_log_marginal_and_posterior_mean(N):
    """The plain method in FP64 (the n = 10^4, p = 5 logistic workload), whole runs on the GPU from
    initialisation to a = 1, ten seeds: the mean log Z within 0.1 of the importance-sampling
    log p(y) and the mean posterior mean within 0.05 posterior sd in every coordinate (Monte
    Carlo error of one run at N = 256 is about 0.3 in log Z and 0.08 sd, hence the seed average;
    N = 2048 repeats the check with smaller spread)."""
    from smc_workloads import logistic_1e4
    wl = logistic_1e4()
    ref = _importance_reference(wl)
    assert ref["rel_se"] < 0.01
    lz, means = [], []
    for seed in range(1, 11):
        z, mean = _plain_run(wl, seed, N)
        lz.append(z - ref["log_ml"])
        means.append((mean - ref["mean"]) / ref["sd"])
    assert abs(np.mean(lz)) < 0.1, lz
    assert np.max(np.abs(np.mean(means, axis=0))) < 0.05, np.mean(means, axis=0)


def test_poisson_gradient_against_finite_differences_at_every_stage():
    """Poisson regression at full size (n = 5e6, p = 50, X in BF16; N = 8192, m = 2000, G = 20,
    L = 20): after each of the first stages from initialisation, and of two stages started from a
    late cloud, the gradient of a*l_hat - a^2/2*sigma2_hat + log p(theta) from loglik_grad at 32
    random particles of the run (their theta, u and the stage's temperature) against central
    differences of the oracle's FP64 estimator on the same stored values, within 1e-4 of the
    largest component."""
    from gpu_common import device_arrays
    from smc_workloads import poisson_5e6
    wl = poisson_5e6("bf16")
    tb = state_round(wl.theta_true, "bf16")
    prob = O.Problem(wl.family, wl.X, wl.y, wl.prior_mean, wl.prior_var)
    prob.set_centre(tb)
    X, y = device_arrays(wl)
    ctx = S().smc_init(X, y, wl.family, wl.prior_mean, wl.prior_var, N=wl.N, m=wl.m, G=wl.G,
                       L=wl.L, seed=wl.seed, ess_frac=0.5, theta_bar=tb)
    del X, y
    rng = np.random.default_rng(32)
    p = wl.p

    def check_stage():
        a = S().smc_get_status(ctx)["a"]
        th, u, _ = S().smc_get_particles(ctx)
        pick = rng.choice(wl.N, size=32, replace=False)
        th_s = th[pick].contiguous()
        u_s = u[pick].contiguous()
        g, _, _ = S().loglik_grad(ctx, th_s, u_s, a)
        thd = th_s.cpu().double().numpy()
        us = u_s.cpu().numpy().astype(np.int64)
        h = 1e-5 * np.maximum(1.0, np.abs(thd))
        pert = np.repeat(thd[:, None, :], 2 * p, axis=1)  # [32, 2p, p]
        for k in range(p):
            pert[:, 2 * k, k] += h[:, k]
            pert[:, 2 * k + 1, k] -= h[:, k]
        ur = np.repeat(us[:, None, :], 2 * p, axis=1)
        r = O.loglik_batch(prob, wl.m, wl.G, pert.reshape(-1, p), ur.reshape(-1, wl.m), grad=False)
        lp = np.array([O.log_prior(t, wl.prior_mean, wl.prior_var)[0]
                       for t in pert.reshape(-1, p)])
        f = (a * r["ell"] - 0.5 * a * a * r["sigma2"] + lp).reshape(32, 2 * p)
        fd = (f[:, 0::2] - f[:, 1::2]) / (2.0 * h)
        gg = g.cpu().double().numpy()
        gs = np.maximum(np.max(np.abs(fd), axis=1, keepdims=True), 1.0)
        err = np.max(np.abs(gg - fd) / gs)
        assert err <= 1e-4, (a, err)
        return a

    temps = []
    for _ in range(4):
        S().smc_reweight(ctx)
        S().smc_resample(ctx)
        S().smc_move(ctx, wl.R)
        temps.append(check_stage())
    # a late cloud: posterior-scale spread around the centre, temperature 0.9
    th = state_round(tb + 2e-4 * rng.standard_normal((wl.N, p)), "bf16")
    u = rng.integers(0, wl.n, size=(wl.N, wl.m)).astype(np.int64)
    S().smc_set_particles(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV))
    S().smc_set_scalars(ctx, 40, 0.9, 0.2, 0.0)
    for _ in range(2):
        S().smc_reweight(ctx)
        S().smc_resample(ctx)
        S().smc_move(ctx, wl.R)
        temps.append(check_stage())
    S().smc_free(ctx)
    assert temps[0] < 1e-3 and temps[-1] > 0.9


def test_nonfinite_particle_is_reported_and_the_context_recovers():
    """A NaN planted in one particle's theta from the host: the cache refresh of smc_set_particles
    flags it and the call returns SMC_ERR_NONFINITE (no trap, no fault); after clean particles are
    set the same context runs a whole stage with finite results."""
    from smc_workloads import small_glm
    wl = small_glm("logistic", n=3000, p=6, N=128, m=40, G=4, L=5, x_dtype="f32", seed=4)
    prob, ctx = make_pair(wl)
    th, u, W = (t.clone() for t in S().smc_get_particles(ctx))
    bad = th.clone()
    bad[17, 3] = float("nan")
    with pytest.raises(S()._abi.SmcError) as ei:
        S().smc_set_particles(ctx, bad, u, W)
    assert ei.value.code == -3
    S().smc_set_particles(ctx, th, u, W)
    ell, s2, _ = S().smc_get_cache(ctx)
    assert torch.isfinite(ell).all() and torch.isfinite(s2).all()
    a, lz, ess = S().smc_reweight(ctx)
    S().smc_resample(ctx)
    acc_u, acc_t = S().smc_move(ctx, 2)
    assert 0.0 < a <= 1.0 and math.isfinite(lz) and math.isfinite(ess)
    assert 0.0 <= acc_u <= 1.0 and 0.0 <= acc_t <= 1.0
    th2, _, _ = S().smc_get_particles(ctx)
    assert torch.isfinite(th2).all()
    S().smc_free(ctx)


@pytest.mark.parametrize("x_dtype", ["bf16", "f32"])
def test_logistic_row_terms_on_every_branch(x_dtype):
    """The per-row increment d_j = l_j - q_j and its eta-derivative r_j (saved by loglik_fwd) for
    particles from 1e-3 to about 10 away from the centre, so D = x'(theta - theta_bar) runs from
    the cumulant series (|D| <= 1/2) through the exp/log form to |D| of about 40: against the
    definitions evaluated in FP64 with numpy on the same stored values,
    d = l(eta) - l(eta_bar) - l'(eta_bar) D - l''(eta_bar) D^2/2 and r = l'(eta) - l'(eta_bar) -
    l''(eta_bar) D. Bars: 2e-6 of the size of the terms d cancels from (|D| + D^2/8) plus 5e-7
    (a warp takes the exp/log form for all its rows once one of them is past the series range,
    and that form errs by about 3e-7 absolute), and 2e-6 of (1 + |D|/4) for r (the FP32 rounding
    of D and eta_bar alone moves d by r dD); rows in warps that stay on the series have no
    absolute term."""
    from scipy import special
    from smc_workloads import small_glm
    wl = small_glm("logistic", n=4000, p=20, N=64, m=192, G=4, L=2, x_dtype=x_dtype, seed=8,
                   theta_scale=0.6)  # m: whole sweeps of 32 rows (one sweep = one warp's rows)
    prob, ctx = make_pair(wl)
    rng = np.random.default_rng(9)
    B = 64
    scales = np.geomspace(1e-3, 10.0, B)
    th = state_round(prob.theta_bar + scales[:, None] * rng.standard_normal((B, wl.p))
                     / math.sqrt(wl.p), x_dtype)
    u = rng.integers(0, wl.n, size=(B, wl.m)).astype(np.int64)
    _, _, d_g, r_g = S().loglik_fwd(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV))
    S().smc_free(ctx)
    d_g, r_g = d_g.cpu().double().numpy(), r_g.cpu().double().numpy()
    Xu = wl.X[u]  # [B, m, p] stored values
    yu = wl.y[u]
    eb = Xu @ prob.theta_bar
    D = np.einsum("bjp,bp->bj", Xu, th - prob.theta_bar[None, :])
    eta = eb + D

    def ell(e):
        return yu * e - np.logaddexp(0.0, e)

    sb = special.expit(eb)
    w = sb * (1.0 - sb)
    d_ref = ell(eta) - ell(eb) - (yu - sb) * D + 0.5 * w * D * D
    r_ref = (yu - special.expit(eta)) - (yu - sb) + w * D
    assert np.abs(D).max() > 20 and np.abs(D).min() < 1e-3
    assert ((np.abs(D) > 0.5) & (np.abs(D) < 2)).sum() > 500  # rows just past the series range
    # warps (32 consecutive rows of a particle's sweep) whose rows all lie in the series range
    series_warp = np.repeat((np.abs(D).reshape(B, -1, 32) <= 0.5).all(axis=2), 32, axis=1)
    absd = np.where(series_warp, 1e-12, 5e-7)
    assert np.all(np.abs(d_g - d_ref) <= 2e-6 * (np.abs(D) + D * D / 8) + absd)
    assert np.all(np.abs(r_g - r_ref) <= 2e-6 * (1.0 + np.abs(D) / 4))
    assert series_warp.any() and (~series_warp).any()
