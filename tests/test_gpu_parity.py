"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the same seeded
inputs. Sizes span several tiles with ragged tails (m not a multiple of the rows per warp step, G
not dividing m, odd p)."""
import math

import numpy as np
import pytest
import torch

from gpu_common import ell_scale, make_pair, oracle_problem, state_round, tol
from oracle import oracle as O
from smc_workloads import small_glm

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def S():
    import paper_1805_03317_gb300 as pkg
    return pkg


def _wl(family, x_dtype, p=7, n=5000, N=64, m=77, G=5, seed=11):
    kw = dict(x_scale=0.3) if family == "poisson" else {}
    return small_glm(family, n=n, p=p, N=N, m=m, G=G, L=4, x_dtype=x_dtype, seed=seed, **kw)


def _particles(prob, B, m, scale, x_dtype, seed=3):
    rng = np.random.default_rng(seed)
    th = state_round(prob.theta_bar + scale * rng.standard_normal((B, prob.p)), x_dtype)
    u = rng.integers(0, prob.n, size=(B, m)).astype(np.int64)
    return th, u


def _check_estimates(x_dtype, got, ref, prob=None, theta=None):
    t = tol(x_dtype)
    ell, s2, g = got
    if prob is None:
        np.testing.assert_allclose(ell, ref["ell"], rtol=t["ell"], atol=0)
    else:  # against the estimator's largest summand (it may nearly cancel)
        assert np.all(np.abs(ell - ref["ell"]) <= t["ell"] * ell_scale(prob, theta, ref["ell"]))
    # sigma2_hat enters the log target additively (-a^2/2 sigma2_hat), so its error is held to its
    # own relative bar plus the bar of l_hat in the same units
    bound = t["sig2"] * np.max(np.abs(ref["sigma2"])) + t["ell"] * np.max(np.abs(ref["ell"]))
    assert np.max(np.abs(s2 - ref["sigma2"])) <= bound
    if g is not None:
        gs = np.maximum(np.max(np.abs(ref["grad"]), axis=1, keepdims=True), 1.0)
        err = np.abs(g - ref["grad"]) / gs
        assert err.max() <= t["grad"], err.max()


@pytest.mark.parametrize("x_dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("family", ["logistic", "poisson", "gaussian", "probit"])
@pytest.mark.parametrize("hint", range(0, 13))
def test_estimator_and_gradient_match_oracle(family, x_dtype, hint):
    wl = _wl(family, x_dtype)
    try:
        prob, ctx = make_pair(wl, tile_hint=hint)
    except S()._abi.SmcError as e:
        if e.code == -1 and hint > 0:
            pytest.skip("tile not compiled for this storage type or too narrow")
        raise
    th, u = _particles(prob, 37, wl.m, 0.1, x_dtype)
    a = 0.8
    g, ell, s2 = S().loglik_grad(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV), a)
    ref = O.loglik_batch(prob, wl.m, wl.G, th, u, a=a)
    _check_estimates(x_dtype, (ell.cpu().numpy(), s2.cpu().numpy(),
                               g.cpu().double().numpy()), ref)
    ell2, s22 = S().loglik_est(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV))
    _check_estimates(x_dtype, (ell2.cpu().numpy(), s22.cpu().numpy(), None), ref)
    S().smc_free(ctx)


@pytest.mark.parametrize("x_dtype", ["f32", "bf16"])
@pytest.mark.parametrize("hint", range(0, 13))
def test_wide_rows_match_oracle(x_dtype, hint):
    """p = 101 (the GAM's width): rows span 13-26 vectors, so only the widest tiles cover them."""
    wl = small_glm("logistic", n=6000, p=101, N=24, m=333, G=10, L=3, x_dtype=x_dtype, seed=5,
                   x_scale=0.1, theta_scale=0.1)
    try:
        prob, ctx = make_pair(wl, tile_hint=hint)
    except S()._abi.SmcError as e:
        if e.code == -1 and hint > 0:
            pytest.skip("tile not compiled for this storage type or too narrow")
        raise
    th, u = _particles(prob, 24, wl.m, 0.05, x_dtype)
    g, ell, s2 = S().loglik_grad(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV), 0.7)
    ref = O.loglik_batch(prob, wl.m, wl.G, th, u, a=0.7)
    _check_estimates(x_dtype, (ell.cpu().numpy(), s2.cpu().numpy(), g.cpu().double().numpy()), ref)
    S().smc_free(ctx)


def test_gam_basis_rows_match_oracle():
    """The GAM workload's own rows (B-spline columns, Gaussian response) at small n."""
    from smc_workloads import gam_1e7
    wl = gam_1e7("bf16", n=20000, N=16, m=400, chunk=20000)
    prob, ctx = make_pair(wl)
    th, u = _particles(prob, 16, wl.m, 0.05, "bf16")
    g, ell, s2 = S().loglik_grad(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV), 1.0)
    ref = O.loglik_batch(prob, wl.m, wl.G, th, u, a=1.0)
    _check_estimates("bf16", (ell.cpu().numpy(), s2.cpu().numpy(), g.cpu().double().numpy()), ref)
    S().smc_free(ctx)


@pytest.mark.parametrize("x_dtype", ["f64", "f32", "bf16"])
def test_control_variate_moments_match_oracle(x_dtype):
    wl = _wl("logistic", x_dtype, n=20011)
    prob, ctx = make_pair(wl)
    tb, A, B, C = S().smc_get_centre(ctx)
    np.testing.assert_array_equal(tb, prob.theta_bar)
    # A and B are FP64 sums; C accumulates 32-row tiles in FP32 for FP32/BF16 storage (exact
    # products of the stored values, rounded per tile), FP64 across tiles
    ctol = 1e-10 if x_dtype == "f64" else 2e-6
    assert A == pytest.approx(prob.A, rel=1e-12)
    np.testing.assert_allclose(B, prob.B, rtol=1e-9, atol=1e-9 * np.abs(prob.B).max())
    np.testing.assert_allclose(C, prob.C, rtol=ctol, atol=ctol * 1e-2 * np.abs(prob.C).max())
    # at another point
    pt = prob.theta_bar + 0.2
    A2, B2, C2 = S().smc_cv_moments(ctx, pt)
    Ar, Br, Cr = O.cv_moments("logistic", prob.X, prob.y, pt)
    assert A2 == pytest.approx(Ar, rel=1e-12)
    np.testing.assert_allclose(C2, Cr, rtol=ctol, atol=ctol * 1e-2 * np.abs(Cr).max())
    S().smc_free(ctx)


@pytest.mark.parametrize("family", ["logistic", "poisson", "probit", "gaussian"])
@pytest.mark.parametrize("p", [3, 20, 50, 101, 120, 126])
def test_tensor_core_moments_match_oracle(family, p):
    """C = X' diag(l'') X on tcgen05 (BF16 storage): against the oracle's direct FP64 sums, and
    against the SIMT moment kernel on the same stored values; n not a multiple of the 128-row
    tile."""
    kw = dict(x_scale=0.3 / math.sqrt(p)) if family == "poisson" else dict(x_scale=1.0 / math.sqrt(p))
    wl = small_glm(family, n=9001, p=p, N=8, m=10, G=2, L=2, x_dtype="bf16", seed=13,
                   theta_scale=0.3, **kw)
    prob, ctx = make_pair(wl)
    pt = prob.theta_bar + 0.05
    A2, B2, C2 = S().smc_cv_moments(ctx, pt)
    Ar, Br, Cr = O.cv_moments(family, prob.X, prob.y, pt, sigma=wl.sigma)
    assert A2 == pytest.approx(Ar, rel=1e-12)
    np.testing.assert_allclose(B2, Br, rtol=1e-9, atol=1e-9 * np.abs(Br).max())
    np.testing.assert_allclose(C2, Cr, rtol=2e-6, atol=2e-8 * np.abs(Cr).max())
    S().smc_free(ctx)
    if p * (p + 1) // 2 > 8192:
        return  # beyond the SIMT kernel's pair slots
    prob2, ctx2 = make_pair(wl, cv_kernel=1)
    A3, B3, C3 = S().smc_cv_moments(ctx2, pt)
    np.testing.assert_allclose(C3, C2, rtol=4e-6, atol=4e-8 * np.abs(Cr).max())
    S().smc_free(ctx2)


@pytest.mark.parametrize("family", ["logistic", "poisson", "probit", "gaussian"])
def test_device_newton_centre_matches_oracle(family):
    wl = _wl(family, "f64", n=8000)
    from gpu_common import device_arrays
    prob = oracle_problem(wl)
    X, y = device_arrays(wl)
    ctx = S().smc_init(X, y, family, wl.prior_mean, wl.prior_var, N=8, m=10, G=2, L=2, seed=1,
                       noise_sigma=wl.sigma, theta_bar=None)
    tb = S().smc_get_centre(ctx)[0]
    np.testing.assert_allclose(tb, prob.theta_bar, rtol=1e-8, atol=1e-10)
    S().smc_free(ctx)


@pytest.mark.parametrize("family,x_dtype", [("logistic", "bf16"), ("poisson", "f32"),
                                            ("probit", "f64")])
def test_device_newton_centre_with_subsample_start_matches_oracle(family, x_dtype):
    """n = 300000: the device Newton first converges on a strided subsample of 75000 rows (sums
    scaled by n / n_sub), then iterates on all rows; the centre is still the full-data posterior
    mode of the stored values."""
    wl = _wl(family, x_dtype, n=300000)
    from gpu_common import device_arrays
    prob = oracle_problem(wl)
    X, y = device_arrays(wl)
    ctx = S().smc_init(X, y, family, wl.prior_mean, wl.prior_var, N=8, m=10, G=2, L=2, seed=1,
                       noise_sigma=wl.sigma, theta_bar=None)
    tb = S().smc_get_centre(ctx)[0]
    np.testing.assert_allclose(tb, state_round(prob.theta_bar, x_dtype), rtol=1e-6, atol=1e-7)
    S().smc_free(ctx)


@pytest.mark.parametrize("x_dtype", ["f64", "f32"])
def test_initial_particles_and_cache_match_oracle(x_dtype):
    wl = _wl("logistic", x_dtype, N=50, m=31, G=4)
    prob, ctx = make_pair(wl)
    th, u, W = S().smc_get_particles(ctx)
    th_o, u_o = O.init_particles(wl.seed, wl.N, wl.p, wl.m, wl.n, wl.prior_mean, wl.prior_var)
    np.testing.assert_array_equal(u.cpu().numpy(), u_o)
    np.testing.assert_allclose(th.cpu().double().numpy(), state_round(th_o, x_dtype), rtol=1e-12,
                               atol=1e-12)
    np.testing.assert_array_equal(W.cpu().numpy(), np.full(wl.N, 1.0 / wl.N))
    ell, s2, blk = S().smc_get_cache(ctx)
    ref = O.loglik_batch(prob, wl.m, wl.G, state_round(th_o, x_dtype), u_o, grad=False,
                         blocks=True)
    _check_estimates(x_dtype, (ell.cpu().numpy(), s2.cpu().numpy(), None), ref)
    rb = ref["blocks"]
    assert np.max(np.abs(blk.cpu().numpy() - rb)) <= tol(x_dtype)["sig2"] * max(1e-300,
                                                                                np.abs(rb).max())
    S().smc_free(ctx)


def _random_cloud(prob, wl, x_dtype, seed=5, spread=0.05):
    rng = np.random.default_rng(seed)
    th = state_round(prob.theta_bar + spread * rng.standard_normal((wl.N, wl.p)), x_dtype)
    u = rng.integers(0, wl.n, size=(wl.N, wl.m)).astype(np.int64)
    W = rng.random(wl.N) ** 3
    W /= W.sum()
    return th, u, W


@pytest.mark.parametrize("x_dtype", ["f64", "f32"])
@pytest.mark.parametrize("a0", [0.0, 0.05, 0.9])
def test_reweight_moments_and_mass_match_oracle(x_dtype, a0):
    wl = _wl("logistic", x_dtype, N=300, m=40, G=4)
    prob, ctx = make_pair(wl)
    th, u, W = _random_cloud(prob, wl, x_dtype)
    S().smc_set_particles(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV),
                          torch.from_numpy(W).to(DEV))
    S().smc_set_scalars(ctx, 4, a0, 0.3, 0.0)
    a_new, lz, ess = S().smc_reweight(ctx)
    ref = O.loglik_batch(prob, wl.m, wl.G, th, u, grad=False)
    ra, rlogW, rW, rlz, ress = O.reweight(np.log(W), ref["ell"], ref["sigma2"], a0, 0.5)
    t = tol(x_dtype)
    rtol = 1e-12 if x_dtype == "f64" else 1e-5
    assert a_new == pytest.approx(ra, rel=rtol, abs=1e-15)
    # log Z increment = LSE(new) - LSE(old): FP64 cancellation leaves ~1e-15 * |log N| absolute
    lz_abs = t["ell"] * abs(ref["ell"]).max() * abs(a_new - a0) + 1e-13
    assert lz == pytest.approx(rlz, rel=rtol, abs=lz_abs)
    assert ess == pytest.approx(ress, rel=max(rtol, 1e-9))
    _, _, Wg = S().smc_get_particles(ctx)
    np.testing.assert_allclose(Wg.cpu().numpy(), rW, rtol=1e-6 if x_dtype != "f64" else 1e-9,
                               atol=1e-12)
    mean, Sig, Lc, rc = O.moments(rW, th)
    Sg, Lg = S().smc_get_mass(ctx)
    np.testing.assert_allclose(Sg, Sig, rtol=1e-9, atol=1e-12 * np.abs(Sig).max())
    np.testing.assert_allclose(Lg, Lc, rtol=1e-8, atol=1e-10 * np.abs(Lc).max())
    S().smc_free(ctx)


def test_first_stage_reweight_with_large_log_weights():
    """Prior particles far from the data: |l_hat| ~ 1e6 and sigma2_hat ~ 1e9 make the candidate log
    weights reach ~1e9 at the first stage; the temperature search must stay finite and agree."""
    from smc_workloads import logistic_1e6
    wl = logistic_1e6("bf16", n=100_000)
    wl.N, wl.m = 512, 1000
    prob, ctx = make_pair(wl, theta_bar=wl.theta_true)
    th_o, u_o = O.init_particles(wl.seed, wl.N, wl.p, wl.m, wl.n, wl.prior_mean, wl.prior_var)
    th_o = state_round(th_o, "bf16")
    S().smc_set_particles(ctx, torch.from_numpy(th_o).to(DEV), torch.from_numpy(u_o).to(DEV))
    ell, s2, _ = S().smc_get_cache(ctx)
    assert float(ell.abs().max()) > 1e5 and float(s2.max()) > 1e6
    a_new, lz, ess = S().smc_reweight(ctx)
    ref = O.loglik_batch(prob, wl.m, wl.G, th_o, u_o, grad=False)
    ra, _, _, rlz, ress = O.reweight(np.full(wl.N, -np.log(wl.N)), ref["ell"], ref["sigma2"], 0.0,
                                     0.5)
    assert np.isfinite(a_new) and np.isfinite(lz) and np.isfinite(ess)
    assert a_new == pytest.approx(ra, rel=1e-4)
    assert ess == pytest.approx(ress, rel=1e-3)
    S().smc_free(ctx)


@pytest.mark.parametrize("N", [1, 7, 300, 5000])
def test_resampling_ancestors_bit_exact(N):
    wl = _wl("logistic", "f64", N=N, m=9, G=3)
    prob, ctx = make_pair(wl)
    rng = np.random.default_rng(N)
    th = prob.theta_bar + 0.1 * rng.standard_normal((N, wl.p))
    u = rng.integers(0, wl.n, size=(N, wl.m)).astype(np.int64)
    W = rng.random(N) ** 6
    W /= W.sum()
    S().smc_set_particles(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV),
                          torch.from_numpy(W).to(DEV))
    stage = 9
    S().smc_set_scalars(ctx, stage, 0.5, 0.3, 0.0)
    anc = torch.empty(N, dtype=torch.int32, device=DEV)
    S().smc_resample(ctx, anc)
    U = O.uniform(O.r64(wl.seed, O.TAG_RESAMPLE, O.stage_move(stage, 0), 0, 0))
    ref = O.resample(W, U)
    np.testing.assert_array_equal(anc.cpu().numpy(), ref)
    th2, u2, W2 = S().smc_get_particles(ctx)
    np.testing.assert_array_equal(th2.cpu().numpy(), th[ref])
    np.testing.assert_array_equal(u2.cpu().numpy(), u[ref])
    np.testing.assert_array_equal(W2.cpu().numpy(), np.full(N, 1.0 / N))
    S().smc_free(ctx)


@pytest.mark.parametrize("hmc_kernel", [1, 0])
def test_moves_match_oracle_fp64(hmc_kernel):
    """One Algorithm-1 move (u block update, then HMC) on identical particles: indices and accept
    decisions bit-exact, theta to FP64 rounding. hmc_kernel 1 = streamed rows, 0 = automatic
    (rows resident in shared memory for this size)."""
    wl = _wl("logistic", "f64", N=200, m=60, G=6)
    prob, ctx = make_pair(wl, hmc_kernel=hmc_kernel)
    th, u, W = _random_cloud(prob, wl, "f64", spread=0.03)
    S().smc_set_particles(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV),
                          torch.from_numpy(W).to(DEV))
    S().smc_set_scalars(ctx, 2, 0.3, 0.4, 0.0)
    a, _, _ = S().smc_reweight(ctx)  # stage 3: also sets the mass matrix from this cloud
    eps = 0.4  # set above; smc_reweight does not change it
    acc_u, acc_t = S().smc_move(ctx, 1)
    th_g, u_g, _ = S().smc_get_particles(ctx)
    # oracle: same cloud, same temperature, same mass matrix inputs (from the oracle's moments)
    ref = O.loglik_batch(prob, wl.m, wl.G, th, u, grad=False)
    ra, _, rW, _, _ = O.reweight(np.log(W), ref["ell"], ref["sigma2"], 0.3, 0.5)
    assert a == pytest.approx(ra, rel=1e-12)
    _, Sig, Lc, _ = O.moments(rW, th)
    th_o, u_o = th.copy(), u.copy()
    au = O.upm_move(prob, wl.m, wl.G, wl.seed, 3, 0, ra, th_o, u_o)
    at = O.hmc_move(prob, wl.m, wl.G, wl.seed, 3, 0, ra, eps, wl.L, Sig, Lc, th_o, u_o)
    np.testing.assert_array_equal(u_g.cpu().numpy(), u_o)
    assert acc_u == pytest.approx(au.mean()) and acc_t == pytest.approx(at.mean())
    np.testing.assert_allclose(th_g.cpu().numpy(), th_o, rtol=1e-9, atol=1e-11)
    ell, s2, _ = S().smc_get_cache(ctx)
    ref2 = O.loglik_batch(prob, wl.m, wl.G, th_o, u_o, grad=False)
    np.testing.assert_allclose(ell.cpu().numpy(), ref2["ell"], rtol=1e-11)
    S().smc_free(ctx)


@pytest.mark.parametrize("hmc_kernel", [1, 0])
def test_full_smc_run_matches_oracle_fp64(hmc_kernel):
    wl = small_glm("logistic", n=4000, p=4, N=128, m=50, G=5, L=6, R=2, x_dtype="f64", seed=21)
    prob, ctx = make_pair(wl, hmc_kernel=hmc_kernel)
    cfg = O.SMCConfig(N=wl.N, m=wl.m, G=wl.G, L=wl.L, R=wl.R, seed=wl.seed, tau=0.5)
    st_o = O.smc_run(prob, cfg)
    runner = S().SubsampledSMC.__new__(S().SubsampledSMC)
    runner.ctx, runner.history = ctx, []
    st = runner.run(wl.R)
    assert st["stage"] == st_o.stage
    np.testing.assert_allclose([h["a"] for h in runner.history], [h["a"] for h in st_o.history],
                               rtol=1e-9)
    assert st["log_z"] == pytest.approx(st_o.log_z, abs=1e-7)
    th, u, _ = S().smc_get_particles(ctx)
    np.testing.assert_array_equal(u.cpu().numpy(), st_o.us)
    np.testing.assert_allclose(th.cpu().numpy(), st_o.thetas, rtol=1e-7, atol=1e-9)
    S().smc_free(ctx)


@pytest.mark.parametrize("x_dtype", ["f32", "bf16"])
@pytest.mark.parametrize("family", ["logistic", "poisson", "probit"])
@pytest.mark.parametrize("hmc_kernel", [1, 3, 5, 6, 8, 10, 11, 14, 21])
def test_moves_reduced_precision_match_oracle(x_dtype, family, hmc_kernel):
    """FP32 arithmetic on FP32/BF16-stored rows against the FP64 oracle on the same stored values:
    the MH decisions may differ only where the FP64 log ratio is within rounding of the uniform;
    accepted end points agree to FP32 leapfrog rounding. hmc_kernel 5, 8 and 11 are resident tiles
    wider than the rows (32, 20 and 40 slots for p = 13), whose slots past p must read zeros; 10 is
    the tensor-core trajectory kernel (BF16 only), here with one 128-row tile (m = 90); 14 and 21
    are the 16-slot tiles with two warps and one warp per CTA (BF16 only)."""
    _moves_reduced_precision(_wl(family, x_dtype, p=13, N=256, m=90, G=6), x_dtype, hmc_kernel)


@pytest.mark.parametrize("family", ["logistic", "poisson", "probit"])
@pytest.mark.parametrize("p", [33, 37, 40])
@pytest.mark.parametrize("hmc_kernel", [1, 11, 18, 25])
def test_moves_two_columns_per_lane_match_oracle(family, p, hmc_kernel):
    """p past one warp's lanes: the 40-slot resident tiles (hmc_kernel 11: four warps, 18: two,
    25: one)
    hold columns l and l + 32 in lane l (momentum draw, mass-matrix and C products, gradient,
    write-back), against the FP64 oracle on the same BF16-stored values, beside the streamed
    kernel (hmc_kernel 1)."""
    _moves_reduced_precision(_wl(family, "bf16", p=p, N=256, m=90, G=6), "bf16", hmc_kernel)


def _moves_reduced_precision(wl, x_dtype, hmc_kernel):
    try:
        prob, ctx = make_pair(wl, hmc_kernel=hmc_kernel)
    except S()._abi.SmcError as e:
        if e.code == -1:
            pytest.skip("resident tile does not cover this p")
        raise
    th, u, W = _random_cloud(prob, wl, x_dtype, spread=0.02)
    S().smc_set_particles(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV),
                          torch.from_numpy(W).to(DEV))
    S().smc_set_scalars(ctx, 2, 0.3, 0.4, 0.0)
    a, _, _ = S().smc_reweight(ctx)
    S().smc_move(ctx, 1)
    th_g, u_g, _ = S().smc_get_particles(ctx)
    ref = O.loglik_batch(prob, wl.m, wl.G, th, u, grad=False)
    ra, _, rW, _, _ = O.reweight(np.log(W), ref["ell"], ref["sigma2"], 0.3, 0.5)
    assert a == pytest.approx(ra, rel=1e-5)
    _, Sig, Lc, _ = O.moments(rW, th)
    th_o, u_o = th.copy(), u.copy()
    O.upm_move(prob, wl.m, wl.G, wl.seed, 3, 0, ra, th_o, u_o)
    O.hmc_move(prob, wl.m, wl.G, wl.seed, 3, 0, ra, 0.4, wl.L, Sig, Lc, th_o, u_o)
    # the FP64 log ratios of the two sides differ by rounding only; decisions agree except when the
    # ratio is within rounding of the uniform, and agreeing particles end at the same point
    u_same = np.all(u_g.cpu().numpy() == u_o, axis=1)
    assert u_same.mean() >= 0.97
    tg = th_g.cpu().double().numpy()
    moved_g = np.any(tg != th, axis=1)
    moved_o = np.any(th_o != th, axis=1)
    agree = (moved_g == moved_o) & u_same
    assert agree.mean() >= 0.95, agree.mean()
    both = moved_g & moved_o & u_same
    assert both.sum() > 10
    np.testing.assert_allclose(tg[both], th_o[both], rtol=2e-4, atol=2e-5)
    S().smc_free(ctx)


def test_autotune_leaves_state_unchanged():
    wl = _wl("logistic", "bf16", p=20, N=500, m=100, G=10)
    prob, ctx = make_pair(wl)
    before = [t.clone() for t in S().smc_get_particles(ctx)] + list(S().smc_get_cache(ctx))
    st0 = S().smc_get_status(ctx)
    tile, hmc = S().smc_autotune(ctx)
    assert tile >= 1 and hmc >= 1
    after = list(S().smc_get_particles(ctx)) + list(S().smc_get_cache(ctx))
    for x, y in zip(before, after):
        assert torch.equal(x, y)
    assert S().smc_get_status(ctx) == st0
    S().smc_free(ctx)


@pytest.mark.parametrize("x_dtype", ["f32", "bf16"])
def test_conjugate_gaussian_log_marginal_on_gpu(x_dtype):
    """Gaussian response: the second-order control variate is exact, so SMC targets the exact
    posterior; the seed-averaged log marginal likelihood matches the closed form."""
    from scipy import stats
    errs = []
    for seed in range(1, 7):
        wl = small_glm("gaussian", n=300, p=3, N=2048, m=8, G=2, L=8, R=3, x_dtype=x_dtype,
                       seed=3, sigma=0.8, prior_var=4.0)
        X, y = wl.X, wl.y
        logml = stats.multivariate_normal(mean=np.zeros(wl.n),
                                          cov=0.64 * np.eye(wl.n) + 4.0 * X @ X.T).logpdf(y)
        Sinv = X.T @ X / 0.64 + np.eye(3) / 4.0
        mu = np.linalg.solve(Sinv, X.T @ y / 0.64)
        prob, ctx = make_pair(wl, theta_bar=mu, seed=seed)
        runner = S().SubsampledSMC.__new__(S().SubsampledSMC)
        runner.ctx, runner.history = ctx, []
        st = runner.run(wl.R)
        errs.append(st["log_z"] - logml)
        th, _, _ = S().smc_get_particles(ctx)
        sd = np.sqrt(np.diag(np.linalg.inv(Sinv)))
        assert np.all(np.abs(th.cpu().double().numpy().mean(0) - mu) < 0.15 * sd)
        S().smc_free(ctx)
    assert abs(np.mean(errs)) < 0.1, errs


def test_edge_cases():
    # p = 1, m = 1, G = 1, N = 1, empty batch, out-of-range index
    wl = small_glm("logistic", n=50, p=1, N=1, m=1, G=1, L=1, x_dtype="f32", seed=2)
    prob, ctx = make_pair(wl)
    e, s = S().loglik_est(ctx, torch.zeros(0, 1, device=DEV), torch.zeros(0, 1, dtype=torch.int32,
                                                                         device=DEV))
    assert e.numel() == 0
    th = torch.tensor([[0.1]], device=DEV)
    ell, s2 = S().loglik_est(ctx, th, torch.tensor([[49]], device=DEV))
    ref = O.loglik_batch(prob, 1, 1, np.array([[np.float32(0.1)]], dtype=np.float64),
                         np.array([[49]]), grad=False)
    assert ell.item() == pytest.approx(ref["ell"][0], rel=1e-5)
    assert abs(s2.item()) <= 1e-5 * abs(ref["ell"][0])  # one row: sum of squared deviations is 0
    with pytest.raises(S()._abi.SmcError) as ei:
        S().loglik_est(ctx, th, torch.tensor([[50]], device=DEV))
    assert ei.value.code == -1
    a, lz, ess = S().smc_reweight(ctx)  # N = 1: ESS is 1 for every increment
    assert a == 1.0 and ess == pytest.approx(1.0)
    S().smc_resample(ctx)
    S().smc_move(ctx, 2)
    S().smc_free(ctx)
    # G = m: every block is one row
    wl = _wl("poisson", "bf16", N=33, m=12, G=12)
    prob, ctx = make_pair(wl)
    ell, s2, blk = S().smc_get_cache(ctx)
    th_o, u_o = O.init_particles(wl.seed, wl.N, wl.p, wl.m, wl.n, wl.prior_mean, wl.prior_var)
    ref = O.loglik_batch(prob, wl.m, wl.G, state_round(th_o, "bf16"), u_o, grad=False,
                         blocks=True)
    th_r = state_round(th_o, "bf16")
    err = np.abs(ell.cpu().numpy() - ref["ell"])
    assert np.all(err <= 1e-5 * ell_scale(prob, th_r, ref["ell"]))
    S().smc_free(ctx)


def test_bad_arguments_are_rejected():
    wl = small_glm("logistic", n=50, p=3, N=4, m=5, G=2, L=1, x_dtype="f32", seed=2)
    from gpu_common import device_arrays
    X, y = device_arrays(wl)
    with pytest.raises(S()._abi.SmcError):
        S().smc_init(X, y, "logistic", wl.prior_mean, wl.prior_var, N=4, m=5, G=6, L=1, seed=1)
    with pytest.raises(S()._abi.SmcError):
        S().smc_init(X, y, "logistic", wl.prior_mean, -wl.prior_var, N=4, m=5, G=2, L=1, seed=1)
    with pytest.raises(S()._abi.SmcError):
        S().smc_init(X, y, "logistic", wl.prior_mean, wl.prior_var, N=4, m=5, G=2, L=0, seed=1)


# ------------------------------------------------------------------------------------------------
# Differentiable estimator: torch.autograd.Function over the forward/backward kernel pair
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("family", ["logistic", "poisson", "probit", "gaussian"])
def test_autograd_backward_matches_finite_differences_fp64(family):
    """FP64 storage: the backward kernel's gradient of a l_hat - a^2/2 sigma2_hat against central
    differences of the forward kernel itself, at 32 random particles; and equal to the fused
    loglik_grad kernel without its prior term."""
    wl = _wl(family, "f64", p=6, n=3000, m=90, G=6)
    prob, ctx = make_pair(wl)
    th, u = _particles(prob, 32, wl.m, 0.05, "f64", seed=8)
    a = 0.7
    theta = torch.from_numpy(th).to(DEV).requires_grad_(True)
    ut = torch.from_numpy(u).to(DEV)
    ell, s2 = S().SubsampledLoglik.apply(theta, ut, ctx)
    (a * ell - 0.5 * a * a * s2).sum().backward()
    g = theta.grad.cpu().numpy()
    h = 1e-5
    fd = np.zeros_like(th)
    for c in range(prob.p):
        tp, tm = th.copy(), th.copy()
        tp[:, c] += h
        tm[:, c] -= h
        ep, sp = S().loglik_est(ctx, torch.from_numpy(tp).to(DEV), ut)
        em, sm_ = S().loglik_est(ctx, torch.from_numpy(tm).to(DEV), ut)
        fp = (a * ep - 0.5 * a * a * sp).cpu().numpy()
        fm = (a * em - 0.5 * a * a * sm_).cpu().numpy()
        fd[:, c] = (fp - fm) / (2 * h)
    scale = np.maximum(np.abs(fd).max(axis=1, keepdims=True), 1.0)
    assert (np.abs(g - fd) / scale).max() < 1e-6
    gk, _, _ = S().loglik_grad(ctx, theta.detach(), ut, a)
    prior = -(th - prob.prior_mean) / prob.prior_var
    np.testing.assert_allclose(g, gk.cpu().numpy() - prior, rtol=1e-9, atol=1e-9 * scale.max())
    S().smc_free(ctx)


@pytest.mark.parametrize("x_dtype", ["f32", "bf16"])
@pytest.mark.parametrize("family", ["logistic", "poisson"])
def test_autograd_backward_matches_oracle(family, x_dtype):
    """FP32/BF16 storage: autograd gradient (upstream gradients a and -a^2/2) against the oracle's
    FP64 gradient minus the prior, and against central differences of the oracle's l_hat and
    sigma2_hat on the same stored values, at 32 random particles."""
    wl = _wl(family, x_dtype, p=9, n=4000, m=150, G=10)
    prob, ctx = make_pair(wl)
    th, u = _particles(prob, 32, wl.m, 0.05, x_dtype, seed=9)
    a = 0.8
    theta = torch.from_numpy(th).to(DEV).float().requires_grad_(True)
    ut = torch.from_numpy(u).to(DEV)
    ell, s2 = S().SubsampledLoglik.apply(theta, ut, ctx)
    ref = O.loglik_batch(prob, wl.m, wl.G, th, u, a=a)
    np.testing.assert_allclose(ell.detach().cpu().numpy(), ref["ell"], rtol=1e-5)
    (a * ell - 0.5 * a * a * s2).sum().backward()
    g = theta.grad.double().cpu().numpy()
    prior = -(th - prob.prior_mean) / prob.prior_var
    gref = ref["grad"] - prior
    scale = np.maximum(np.abs(gref).max(axis=1, keepdims=True), 1.0)
    assert (np.abs(g - gref) / scale).max() < 1e-4
    h = 1e-6
    fd = np.zeros_like(th)
    for c in range(prob.p):
        tp, tm = th.copy(), th.copy()
        tp[:, c] += h
        tm[:, c] -= h
        rp = O.loglik_batch(prob, wl.m, wl.G, tp, u, grad=False)
        rm = O.loglik_batch(prob, wl.m, wl.G, tm, u, grad=False)
        fd[:, c] = ((a * rp["ell"] - 0.5 * a * a * rp["sigma2"])
                    - (a * rm["ell"] - 0.5 * a * a * rm["sigma2"])) / (2 * h)
    assert (np.abs(g - fd) / scale).max() < 1e-4
    S().smc_free(ctx)


# ------------------------------------------------------------------------------------------------
# Whole stages as CUDA graphs
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("hmc_kernel", [0, 1])
def test_graph_stages_are_bit_identical(hmc_kernel):
    """smc_stage with graphs (captured at both buffer parities, then replayed), mixed with
    launch-by-launch stages, gives bit-identical particles, weights and log Z to the plain path."""
    wl = _wl("logistic", "bf16", p=7, n=6000, N=300, m=77, G=5)
    _, ca = make_pair(wl, hmc_kernel=hmc_kernel)
    _, cb = make_pair(wl, hmc_kernel=hmc_kernel)
    plan = [True, True, True, False, True, True, False, False, True]
    for use_graph in plan:
        S().smc_stage(ca, 3, use_graph=use_graph)
        S().smc_reweight(cb)
        S().smc_resample(cb)
        S().smc_move(cb, 3)
    ta, ua, Wa = S().smc_get_particles(ca)
    tb_, ub, Wb = S().smc_get_particles(cb)
    assert torch.equal(ta, tb_) and torch.equal(ua, ub) and torch.equal(Wa, Wb)
    sa, sb = S().smc_get_status(ca), S().smc_get_status(cb)
    assert sa == sb
    ea, qa, _ = S().smc_get_cache(ca)
    eb, qb, _ = S().smc_get_cache(cb)
    assert torch.equal(ea, eb) and torch.equal(qa, qb)
    S().smc_free(ca)
    S().smc_free(cb)


# ------------------------------------------------------------------------------------------------
# Full-data comparison method on the tensor cores
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("family", ["logistic", "poisson", "probit", "gaussian"])
@pytest.mark.parametrize("p", [5, 20, 64])
def test_full_data_loglik_matches_oracle(family, p):
    """loglik_full (tcgen05 linear predictor and gradient contraction) against the oracle's direct
    FP64 sums over all rows, for 200 particles (two particle tiles, ragged) and n = 3001 rows (a
    ragged last row tile)."""
    kw = dict(x_scale=0.3 / math.sqrt(p)) if family == "poisson" else dict(x_scale=1.0 / math.sqrt(p))
    wl = small_glm(family, n=3001, p=p, N=8, m=10, G=2, L=2, x_dtype="bf16", seed=21,
                   theta_scale=0.3, **kw)
    prob, ctx = make_pair(wl)
    rng = np.random.default_rng(4)
    B = 200
    th = state_round(prob.theta_bar + 0.1 * rng.standard_normal((B, p)), "bf16")
    a = 0.6
    g, ell = S().loglik_full(ctx, torch.from_numpy(th).to(DEV), a)
    ell = ell.cpu().numpy()
    g = g.double().cpu().numpy()
    for i in range(B):
        lr, gr = O.full_loglik(family, prob.X, prob.y, th[i], sigma=wl.sigma)
        gr = a * gr - (th[i] - prob.prior_mean) / prob.prior_var
        assert abs(ell[i] - lr) <= 1e-5 * abs(lr), (i, ell[i], lr)
        assert np.max(np.abs(g[i] - gr)) <= 1e-4 * max(np.max(np.abs(gr)), 1.0), i
    S().smc_free(ctx)


def test_full_data_smc_recovers_conjugate_posterior():
    """The full-data comparison SMC (exact log-likelihood, tensor-core forces, leapfrog loop as a
    CUDA graph) on the conjugate Gaussian model: the seed-averaged log marginal likelihood and the
    posterior mean match the closed form; graph-captured stages give the same result bit for bit."""
    from scipy import stats
    errs = []
    for seed in range(1, 5):
        wl = small_glm("gaussian", n=300, p=3, N=2048, m=1, G=1, L=8, R=3, x_dtype="bf16",
                       seed=3, sigma=0.8, prior_var=4.0)
        X, y = wl.X, wl.y
        logml = stats.multivariate_normal(mean=np.zeros(wl.n),
                                          cov=0.64 * np.eye(wl.n) + 4.0 * X @ X.T).logpdf(y)
        Sinv = X.T @ X / 0.64 + np.eye(3) / 4.0
        mu = np.linalg.solve(Sinv, X.T @ y / 0.64)
        prob, ctx = make_pair(wl, theta_bar=mu, seed=seed, full_data=True)
        ell, s2, _ = S().smc_get_cache(ctx)
        th0, _, _ = S().smc_get_particles(ctx)
        for i in range(3):
            lr = O.full_loglik("gaussian", prob.X, prob.y, th0[i].double().cpu().numpy(),
                               sigma=wl.sigma, grad=False)
            assert abs(ell[i].item() - lr) <= 1e-5 * abs(lr)
        assert float(s2.abs().max()) == 0.0
        a, stages, acc = 0.0, 0, []
        while a < 1.0 and stages < 200:
            a, _, _ = S().smc_reweight(ctx)
            S().smc_resample(ctx)
            acc.append(S().smc_move(ctx, wl.R)[1])
            stages += 1
        st = S().smc_get_status(ctx)
        errs.append(st["log_z"] - logml)
        assert np.mean(acc) > 0.3, acc
        th, _, _ = S().smc_get_particles(ctx)
        sd = np.sqrt(np.diag(np.linalg.inv(Sinv)))
        assert np.all(np.abs(th.cpu().double().numpy().mean(0) - mu) < 0.15 * sd)
        S().smc_free(ctx)
    assert abs(np.mean(errs)) < 0.1, errs


def test_full_data_graph_stages_are_bit_identical():
    wl = small_glm("logistic", n=4000, p=9, N=256, m=1, G=1, L=5, x_dtype="bf16", seed=6)
    _, ca = make_pair(wl, full_data=True)
    _, cb = make_pair(wl, full_data=True)
    for use_graph in [True, True, False, True]:
        S().smc_stage(ca, 2, use_graph=use_graph)
        S().smc_reweight(cb)
        S().smc_resample(cb)
        S().smc_move(cb, 2)
    ta, _, Wa = S().smc_get_particles(ca)
    tb_, _, Wb = S().smc_get_particles(cb)
    assert torch.equal(ta, tb_) and torch.equal(Wa, Wb)
    assert S().smc_get_status(ca) == S().smc_get_status(cb)
    S().smc_free(ca)
    S().smc_free(cb)


# ------------------------------------------------------------------------------------------------
# Batches of independent posteriors of uneven n and p
# ------------------------------------------------------------------------------------------------
def _batch_problem_dicts(wls):
    from gpu_common import device_arrays
    out = []
    for w in wls:
        X, y = device_arrays(w)
        out.append(dict(X=X, y=y, family=w.family, prior_mean=w.prior_mean, prior_var=w.prior_var,
                        N=w.N, m=w.m, G=w.G, L=w.L, seed=w.seed))
    return out


@pytest.mark.parametrize("streamed,n_lo,n_hi",
                         [(False, 2000, 20000), (False, 300000, 1000000), (True, 2000, 20000)])
def test_batch_stages_match_single_problems(streamed, n_lo, n_hi):
    """One batched u-update launch per move and one trajectory launch per group, the groups side
    by side on side streams (resident tiles grouped by p and by warps per CTA: one or two for
    small subsamples, four above 512 rows; the streamed kernel when asked; the stage steps of all
    problems in shared launches; plain and graph-replayed stages) give bit-identical results to
    stepping each problem alone with the same tiles. n in [2000, 20000] gives m = 100 everywhere, [3e5, 1e6] a mix of
    m = 337 .. 725."""
    from smc_workloads import batch_uneven
    wls = batch_uneven(P=7, N=96, G=5, L=4, R=2, n_lo=n_lo, n_hi=n_hi)
    dicts = _batch_problem_dicts(wls)
    if streamed:
        for d in dicts:
            d["hmc_kernel"] = 1
    b = S().smc_batch_init(dicts)
    tile = S().smc_batch_tile(b)
    kernels = [S().smc_batch_hmc_kernel(b, q) for q in range(len(wls))]
    if streamed:
        assert kernels == [1] * len(wls)
    else:
        # every p here (5..40) has a resident tile; p > 32 takes a 40-slot two-column tile, with
        # one warp per CTA up to m = 160 (hmc_kernel 25), two up to m = 512 (18), four above (11)
        assert len(set(kernels)) >= 3 and all(k >= 2 for k in kernels)
        assert any(w.p > 32 for w in wls)
        assert all(k == (25 if w.m <= 160 else 18 if w.m <= 512 else 11)
                   for k, w in zip(kernels, wls) if w.p > 32)
        if n_hi > 100000:
            assert any(w.m > 512 for w in wls) and any(w.m <= 512 for w in wls)
    # the singles take the batch problems' centres (the device's Newton modes)
    singles = [make_pair(w, tile_hint=tile, hmc_kernel=kernels[q],
                         theta_bar=S().smc_get_centre(S().smc_batch_context(b, q))[0])[1]
               for q, w in enumerate(wls)]
    for use_graph in [False, True, True, False, True, True]:
        S().smc_batch_stage(b, 2, use_graph=use_graph)
        for c in singles:
            S().smc_reweight(c)
            S().smc_resample(c)
            S().smc_move(c, 2)
    for q, c in enumerate(singles):
        cb = S().smc_batch_context(b, q)
        ta, ua, Wa = S().smc_get_particles(cb)
        ts, us, Ws = S().smc_get_particles(c)
        assert torch.equal(ta, ts) and torch.equal(ua, us) and torch.equal(Wa, Ws), q
        assert S().smc_get_status(cb) == S().smc_get_status(c), q
        S().smc_free(c)
    S().smc_batch_free(b)


def test_batch_autotune_leaves_state_unchanged():
    from smc_workloads import batch_uneven
    wls = batch_uneven(P=4, N=64, G=5, L=3, R=2, n_lo=2000, n_hi=10000, seed_offset=1)
    b = S().smc_batch_init(_batch_problem_dicts(wls))
    S().smc_batch_stage(b, 2, use_graph=False)
    before = [S().smc_get_particles(S().smc_batch_context(b, q)) for q in range(4)]
    tile = S().smc_batch_autotune(b)
    assert tile >= 1
    after = [S().smc_get_particles(S().smc_batch_context(b, q)) for q in range(4)]
    for x, y_ in zip(before, after):
        assert all(torch.equal(u, v) for u, v in zip(x, y_))
    S().smc_batch_stage(b, 2, use_graph=True)
    S().smc_batch_free(b)


@pytest.mark.parametrize("x_dtype", ["f32", "bf16"])
@pytest.mark.parametrize("hmc_kernel", [0, 1])
def test_short_logistic_series_near_centre(x_dtype, hmc_kernel):
    """Particles close to the centre (every |x'(theta - theta_bar)| <= 1/20, so whole warps take the
    four-term cumulant series): estimator, gradient and one HMC move against the oracle."""
    wl = _wl("logistic", x_dtype, p=9, n=5000, N=64, m=150, G=5)
    prob, ctx = make_pair(wl, hmc_kernel=hmc_kernel)
    th, u = _particles(prob, 64, wl.m, 0.002, x_dtype, seed=12)
    D = np.abs((prob.X[u] * (th - prob.theta_bar)[:, None, :]).sum(-1))
    assert D.max() <= 0.05
    g, ell, s2 = S().loglik_grad(ctx, torch.from_numpy(th).to(DEV), torch.from_numpy(u).to(DEV), 0.9)
    ref = O.loglik_batch(prob, wl.m, wl.G, th, u, a=0.9)
    _check_estimates(x_dtype, (ell.cpu().numpy(), s2.cpu().numpy(), g.cpu().double().numpy()), ref)
    S().smc_free(ctx)
