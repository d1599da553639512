"""Pins for the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one oracle routine against the paper's mathematics or an independent source:
published Philox vectors, scipy log-densities, finite differences, exact enumeration of the
difference estimator over all index tuples, closed-form conjugate posteriors, and invariants of
resampling and reweighting. A plausible slip in the oracle (a dropped term, a wrong sign or index,
a transposed operand, a wrong n/m factor) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import special, stats

from oracle import oracle as O
from smc_workloads import small_glm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def scipy_loglik_rows(fam, eta, y, sigma=1.0):
    """Per-row log-densities from scipy's distributions (independent of the oracle)."""
    if fam == "logistic":
        return stats.bernoulli.logpmf(y, special.expit(eta))
    if fam == "poisson":
        return stats.poisson.logpmf(y, np.exp(eta))
    if fam == "gaussian":
        return stats.norm.logpdf(y, loc=eta, scale=sigma)
    if fam == "probit":
        return special.log_ndtr((2 * y - 1) * eta)
    if fam == "student_t":
        return stats.t.logpdf(y, df=5.0, loc=eta, scale=sigma)
    raise ValueError(fam)


def scipy_loglik(fam, X, y, theta, sigma=1.0):
    return float(np.sum(scipy_loglik_rows(fam, X @ theta, y, sigma)))


def scipy_log_prior(theta, mu, var):
    return float(np.sum(stats.norm.logpdf(theta, loc=mu, scale=np.sqrt(var))))


def tiny_problem(fam, n=7, p=3, seed=3, sigma=0.7):
    rng = np.random.default_rng(seed)
    X = np.column_stack([np.ones(n), rng.standard_normal((n, p - 1))])
    t = 0.4 * rng.standard_normal(p)
    eta = X @ t
    if fam == "logistic":
        y = (rng.random(n) < special.expit(eta)).astype(float)
    elif fam == "probit":
        y = (rng.random(n) < special.ndtr(eta)).astype(float)
    elif fam == "poisson":
        y = rng.poisson(np.exp(eta)).astype(float)
    elif fam == "student_t":
        y = eta + sigma * rng.standard_t(5.0, size=n)
    else:
        y = eta + sigma * rng.standard_normal(n)
    prob = O.Problem(fam, X, y, np.zeros(p), np.full(p, 3.0), sigma=sigma)
    prob.set_centre(t + 0.05 * rng.standard_normal(p))
    return prob


# ----------------------------------------------------------------------------------------------
# Random numbers
# ----------------------------------------------------------------------------------------------
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(h, 16) for h in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_index_is_floor_of_scaled_draw_and_uniform():
    seed = 12345
    for j in range(50):
        r = O.r64(seed, O.TAG_INIT_U, 7, 3, j)
        for n in (1, 10, 1_000_003, 5_000_000, (1 << 40) + 17):
            assert O.index(r, n) == (r * n) >> 64  # exact big-integer arithmetic
    counts = np.zeros(10)
    for j in range(20000):
        counts[O.index(O.r64(seed, O.TAG_INIT_U, 0, 1, j), 10)] += 1
    chi2 = float(np.sum((counts - 2000.0) ** 2 / 2000.0))
    assert chi2 < stats.chi2.ppf(0.999, 9)
    u = np.array([O.uniform(O.r64(seed, O.TAG_MH_U, 0, 2, j)) for j in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_draws_are_two_words_of_one_philox_block():
    seed = (0xDEADBEEF << 32) | 0x12345678
    out = O.philox4x32_10([3, 11, (5 << 8) | 2, O.TAG_UPM_IDX], [0x12345678, 0xDEADBEEF])
    r6 = O.r64(seed, O.TAG_UPM_IDX, (5 << 8) | 2, 11, 6)
    r7 = O.r64(seed, O.TAG_UPM_IDX, (5 << 8) | 2, 11, 7)
    assert r6 == (int(out[1]) << 32) | int(out[0])
    assert r7 == (int(out[3]) << 32) | int(out[2])


def test_box_muller_normals_moments():
    z = np.array([O.normal(99, O.TAG_MOMENTUM, 1, i % 97, i // 97) for i in range(40000)])
    assert abs(z.mean()) < 4 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3


# ----------------------------------------------------------------------------------------------
# Families (Sec. 3.1) against scipy, derivatives against finite differences
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("fam", ["logistic", "poisson", "gaussian", "probit", "student_t"])
def test_family_logdensity_and_derivatives(fam):
    sigma = 0.7
    ys = {"logistic": [0.0, 1.0], "probit": [0.0, 1.0], "poisson": [0.0, 1.0, 4.0, 17.0],
          "gaussian": [-1.3, 0.0, 2.5], "student_t": [-1.3, 0.0, 2.5, 40.0]}[fam]
    etas = np.linspace(-6, 6, 25)
    if fam == "probit":
        etas = np.concatenate([etas, [-40.0, -12.0, -5.5, 8.0, 30.0]])
    h = 1e-5
    for y in ys:
        for eta in etas:
            l, d1, d2 = O.family(fam, eta, y, sigma)
            ref = float(scipy_loglik_rows(fam, np.array([eta]), np.array([y]), sigma)[0])
            assert l == pytest.approx(ref, rel=1e-12, abs=1e-12)
            lp, d1p, _ = O.family(fam, eta + h, y, sigma)
            lm, d1m, _ = O.family(fam, eta - h, y, sigma)
            assert d1 == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-7)
            assert d2 == pytest.approx((d1p - d1m) / (2 * h), rel=1e-6, abs=1e-7)


def test_erfcx_continued_fraction():
    for x in np.linspace(3.0, 60.0, 40):
        assert O.lib().orc_erfcx_cf(x) == pytest.approx(float(special.erfcx(x)), rel=1e-13)


# ----------------------------------------------------------------------------------------------
# Control-variate moments (Sec. 3.2)
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("fam", ["logistic", "poisson", "gaussian", "probit", "student_t"])
def test_cv_moments_against_full_likelihood(fam):
    prob = tiny_problem(fam)
    tb = prob.theta_bar
    assert prob.A == pytest.approx(scipy_loglik(fam, prob.X, prob.y, tb, prob.sigma), rel=1e-13)
    h = 1e-5
    for c in range(prob.p):
        e = np.zeros(prob.p)
        e[c] = h
        fd = (scipy_loglik(fam, prob.X, prob.y, tb + e, prob.sigma)
              - scipy_loglik(fam, prob.X, prob.y, tb - e, prob.sigma)) / (2 * h)
        assert prob.B[c] == pytest.approx(fd, rel=1e-6, abs=1e-7)
        _, Bp, _ = O.cv_moments(fam, prob.X, prob.y, tb + e, prob.sigma)
        _, Bm, _ = O.cv_moments(fam, prob.X, prob.y, tb - e, prob.sigma)
        np.testing.assert_allclose(prob.C[:, c], (Bp - Bm) / (2 * h), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(prob.C, prob.C.T, rtol=0, atol=1e-13)


@pytest.mark.parametrize("fam", ["logistic", "poisson", "probit", "student_t"])
def test_moment_identity_sum_of_row_control_variates(fam):
    """sum_k q_k(theta) built row by row equals A + B'delta + delta'C delta/2 (Sec. 3.2)."""
    prob = tiny_problem(fam, n=9)
    rng = np.random.default_rng(5)
    theta = prob.theta_bar + 0.3 * rng.standard_normal(prob.p)
    d = theta - prob.theta_bar
    total = 0.0
    for k in range(prob.n):
        Ak, Bk, Ck = O.cv_moments(fam, prob.X[k:k + 1], prob.y[k:k + 1], prob.theta_bar,
                                  prob.sigma)
        total += Ak + Bk @ d + 0.5 * d @ Ck @ d
    assert total == pytest.approx(prob.A + prob.B @ d + 0.5 * d @ prob.C @ d, rel=1e-12)


# ----------------------------------------------------------------------------------------------
# Difference estimator (Eq. difference_estimator_logl) and variance estimate
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("fam", ["logistic", "poisson", "probit", "student_t"])
def test_estimator_unbiased_by_enumeration(fam):
    """Averaging l_hat over all n^m equally likely index tuples gives l(theta) exactly; and the
    printed sigma2_hat has expectation (m-1)/m * Var(l_hat) (sampling with replacement)."""
    n, m = 5, 3
    prob = tiny_problem(fam, n=n, p=2, seed=11)
    theta = prob.theta_bar + np.array([0.4, -0.7])
    us = np.array([[a, b, c] for a in range(n) for b in range(n) for c in range(n)],
                  dtype=np.int64)
    thetas = np.repeat(theta[None, :], us.shape[0], axis=0)
    out = O.loglik_batch(prob, m, 1, thetas, us, a=1.0, grad=False)
    exact = scipy_loglik(fam, prob.X, prob.y, theta, prob.sigma)
    assert out["ell"].mean() == pytest.approx(exact, rel=1e-12)
    var = out["ell"].var()
    assert out["sigma2"].mean() == pytest.approx((m - 1) / m * var, rel=1e-10)
    assert var > 1e-6  # the check above is not vacuous


@pytest.mark.parametrize("fam", ["logistic", "poisson", "probit", "student_t"])
def test_target_gradient_finite_difference(fam):
    """The HMC force is the gradient of a*l_hat - a^2/2*sigma2_hat + log p(theta) for fixed u."""
    prob = tiny_problem(fam, n=40, p=3, seed=4)
    rng = np.random.default_rng(8)
    m, a = 12, 0.7
    u = rng.integers(0, prob.n, size=(1, m)).astype(np.int64)
    theta = prob.theta_bar + 0.5 * rng.standard_normal(prob.p)

    def target(t):
        o = O.loglik_batch(prob, m, 3, t[None, :], u, a=a, grad=False)
        return (a * o["ell"][0] - 0.5 * a * a * o["sigma2"][0]
                + scipy_log_prior(t, prob.prior_mean, prob.prior_var))

    g = O.loglik_batch(prob, m, 3, theta[None, :], u, a=a)["grad"][0]
    h = 1e-6
    for c in range(prob.p):
        e = np.zeros(prob.p)
        e[c] = h
        fd = (target(theta + e) - target(theta - e)) / (2 * h)
        assert g[c] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_estimator_at_centre_and_gaussian_exactness():
    prob = tiny_problem("logistic", n=30)
    rng = np.random.default_rng(2)
    u = rng.integers(0, prob.n, size=(1, 10)).astype(np.int64)
    a = 0.3
    o = O.loglik_batch(prob, 10, 2, prob.theta_bar[None, :], u, a=a)
    assert o["ell"][0] == pytest.approx(prob.A, rel=1e-14)
    assert o["sigma2"][0] == pytest.approx(0.0, abs=1e-20)
    gp = -(prob.theta_bar - prob.prior_mean) / prob.prior_var
    np.testing.assert_allclose(o["grad"][0], a * prob.B + gp, rtol=1e-13, atol=1e-13)
    # Gaussian response: the second-order expansion is exact, so every d_k = 0
    g = tiny_problem("gaussian", n=30)
    theta = g.theta_bar + rng.standard_normal(g.p)
    o = O.loglik_batch(g, 10, 2, theta[None, :], u, a=1.0)
    assert o["ell"][0] == pytest.approx(scipy_loglik("gaussian", g.X, g.y, theta, g.sigma),
                                        rel=1e-12)
    assert abs(o["sigma2"][0]) < 1e-12 * abs(o["ell"][0]) ** 2


def test_block_partials_follow_floor_partition():
    prob = tiny_problem("logistic", n=25, seed=9)
    rng = np.random.default_rng(3)
    m, G = 13, 4
    theta = prob.theta_bar + 0.6 * rng.standard_normal(prob.p)
    u = rng.integers(0, prob.n, size=m).astype(np.int64)
    d_all = []
    q_tot = None
    for k in u:  # per-row d_k from a subsample of size one: l_hat = q(theta) + n*d_k
        o1 = O.loglik_batch(prob, 1, 1, theta[None, :], np.array([[k]]), grad=False)
        dlt = theta - prob.theta_bar
        q_tot = prob.A + prob.B @ dlt + 0.5 * dlt @ prob.C @ dlt
        d_all.append((o1["ell"][0] - q_tot) / prob.n)
    d_all = np.array(d_all)
    o = O.loglik_batch(prob, m, G, theta[None, :], u[None, :], grad=False, blocks=True)
    for g in range(G):
        lo, hi = (g * m) // G, ((g + 1) * m) // G
        assert o["blocks"][0, g, 0] == pytest.approx(d_all[lo:hi].sum(), rel=1e-9, abs=1e-12)
        assert o["blocks"][0, g, 1] == pytest.approx((d_all[lo:hi] ** 2).sum(), rel=1e-9,
                                                     abs=1e-15)
    S, Q = o["blocks"][0, :, 0].sum(), o["blocks"][0, :, 1].sum()
    assert o["sigma2"][0] == pytest.approx(prob.n ** 2 / m ** 2 * (Q - S * S / m), rel=1e-8)
    assert o["ell"][0] == pytest.approx(q_tot + prob.n / m * S, rel=1e-12)


# ----------------------------------------------------------------------------------------------
# Reweighting, ESS and the temperature search (Sec. 2.2, Sec. 3.3, Algorithm 2 (b)-(c))
# ----------------------------------------------------------------------------------------------
def _weights_case(N=300, seed=1):
    rng = np.random.default_rng(seed)
    logW = np.full(N, -math.log(N))
    ell = -5000.0 + 40.0 * rng.standard_normal(N)
    sig2 = np.abs(2.0 + rng.standard_normal(N))
    return logW, ell, sig2


@pytest.mark.parametrize("K", [2, 16])
def test_reweight_bracket_and_log_z(K):
    logW, ell, sig2 = _weights_case()
    N, a, tau = logW.size, 0.2, 0.5
    a_new, lw, W, lz, ess = O.reweight(logW, ell, sig2, a, tau, K=K, rounds=40 if K == 2 else 10)
    D = a_new - a
    assert 0 < D < 1 - a
    inc = D * ell - 0.5 * ((a + D) ** 2 - a ** 2) * sig2
    w = np.exp(logW + inc - np.max(logW + inc))
    Wd = w / w.sum()
    assert ess == pytest.approx(1.0 / np.sum(Wd ** 2), rel=1e-9)  # ESS = (sum W^2)^-1
    assert ess >= tau * N
    width = (1 - a) * K ** -(40 if K == 2 else 10)
    assert O.ess_at(logW, ell, sig2, a, D + 2 * width) < tau * N
    np.testing.assert_allclose(W, Wd, rtol=1e-9, atol=1e-300)
    # log Z increment = log sum_i W_i^{old} * exp(increment_i)   (Sec. 3.5)
    mx = np.max(inc)
    assert lz == pytest.approx(mx + math.log(np.sum(np.exp(logW) * np.exp(inc - mx))), rel=1e-12)


def test_reweight_jumps_to_one_when_ess_allows():
    N = 100
    logW = np.full(N, -math.log(N))
    ell = np.full(N, -10.0) + 1e-3 * np.arange(N)
    sig2 = np.zeros(N)
    a_new, lw, W, lz, ess = O.reweight(logW, ell, sig2, 0.4, 0.5)
    assert a_new == 1.0
    assert ess > 0.99 * N


def test_bisection_and_16ary_agree():
    logW, ell, sig2 = _weights_case(seed=4)
    a2 = O.reweight(logW, ell, sig2, 0.0, 0.5, K=2, rounds=45)[0]
    a16 = O.reweight(logW, ell, sig2, 0.0, 0.5, K=16, rounds=12)[0]
    assert a2 == pytest.approx(a16, rel=1e-11, abs=1e-14)


def _ess_numpy(logW, ell, sig2, a, D):
    lw = logW + D * ell - 0.5 * ((a + D) ** 2 - a ** 2) * sig2
    return float(np.exp(2 * special.logsumexp(lw) - special.logsumexp(2 * lw)))


@pytest.mark.parametrize("a", [0.0, 0.2, 0.9])
def test_grid_rule_takes_the_point_closest_to_the_target(a):
    """The paper's rule (Sec. 2.3): among the grid points the increment whose ESS is closest to
    the target. The grid and the ESS are rebuilt here with numpy and scipy's logsumexp."""
    logW, ell, sig2 = _weights_case(seed=5)
    N, tau, S, E = logW.size, 0.8, 257, 12.0
    a_new, lw, W, lz, ess = O.reweight_grid(logW, ell, sig2, a, tau, S, E)
    dmax = 1.0 - a
    grid = dmax * np.power(10.0, -E * (S - 1 - np.arange(S)) / (S - 1))
    grid[-1] = dmax
    dist = np.array([abs(_ess_numpy(logW, ell, sig2, a, D) - tau * N) for D in grid])
    best = int(np.argmin(dist))
    D = dmax if a_new == 1.0 else a_new - a
    assert D == pytest.approx(grid[best], rel=1e-13)
    assert ess == pytest.approx(_ess_numpy(logW, ell, sig2, a, D), rel=1e-9)
    # the grid is fine enough here that the chosen ESS is near the target (not just the closest)
    assert abs(ess - tau * N) < 0.02 * N
    inc = D * ell - 0.5 * ((a + D) ** 2 - a ** 2) * sig2
    assert lz == pytest.approx(special.logsumexp(logW + inc) - special.logsumexp(logW), rel=1e-12)
    np.testing.assert_allclose(W, np.exp(logW + inc - special.logsumexp(logW + inc)), rtol=1e-9)


def test_grid_rule_takes_one_when_every_point_is_above_the_target():
    N = 100
    logW = np.full(N, -math.log(N))
    ell = np.full(N, -10.0) + 1e-3 * np.arange(N)
    a_new, _, _, _, ess = O.reweight_grid(logW, ell, np.zeros(N), 0.4, 0.8, 64, 8.0)
    assert a_new == 1.0 and ess > 0.99 * N


# ----------------------------------------------------------------------------------------------
# Moments, mass matrix and resampling (Algorithm 2 (d)-(e))
# ----------------------------------------------------------------------------------------------
def test_weighted_moments_against_numpy():
    rng = np.random.default_rng(6)
    N, p = 500, 4
    th = rng.standard_normal((N, p)) @ rng.standard_normal((p, p))
    W = rng.random(N)
    W /= W.sum()
    mean, S, Lc, rc = O.moments(W, th)
    assert rc == 0
    np.testing.assert_allclose(mean, np.average(th, axis=0, weights=W), rtol=1e-12)
    np.testing.assert_allclose(S, np.cov(th.T, aweights=W, ddof=0), rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(Lc, np.linalg.cholesky(S), rtol=1e-10, atol=1e-14)


def test_resampling_invariants():
    rng = np.random.default_rng(7)
    N = 257
    W = rng.random(N) ** 4
    W /= W.sum()
    for U in (0.0, 0.3, 0.999999):
        anc = O.resample(W, U)
        assert np.all(np.diff(anc) >= 0) and anc.min() >= 0 and anc.max() < N
        wq = np.floor(W * 2.0 ** 40)
        exp_count = N * wq / wq.sum()
        counts = np.bincount(anc, minlength=N)
        assert np.all(counts >= np.floor(exp_count)) and np.all(counts <= np.ceil(exp_count))
    np.testing.assert_array_equal(O.resample(np.full(N, 1.0 / N), 0.5), np.arange(N))
    one = np.zeros(N)
    one[17] = 1.0
    np.testing.assert_array_equal(O.resample(one, 0.25), np.full(N, 17))


def test_multinomial_resampling_is_the_inverse_quantised_cdf():
    """Multinomial resampling (Sec. 2.2): each offspring inverts the CDF of the integer weights at
    its own uniform (rebuilt here with numpy's searchsorted); counts over many replications follow
    the multinomial law (mean N w, variance N w (1 - w)), unlike systematic resampling."""
    rng = np.random.default_rng(12)
    N = 211
    W = rng.random(N) ** 4
    W /= W.sum()
    wq = np.floor(W * 2.0 ** 40).astype(np.uint64)
    cum = np.cumsum(wq)
    T = int(cum[-1])
    U = rng.random(N)
    U[:3] = [0.0, 0.5, 1.0 - 2.0 ** -53]
    anc = O.resample_multinomial(W, U)
    pos = np.minimum(np.floor(U * float(T)).astype(np.uint64), np.uint64(T - 1))
    np.testing.assert_array_equal(anc, np.searchsorted(cum, pos, side="right"))
    reps = 3000
    counts = np.zeros((reps, N))
    for r in range(reps):
        counts[r] = np.bincount(O.resample_multinomial(W, rng.random(N)), minlength=N)
    q = wq / float(T)
    mean, var = counts.mean(axis=0), counts.var(axis=0)
    assert np.all(np.abs(mean - N * q) < 5 * np.sqrt(N * q * (1 - q) / reps) + 1e-12)
    big = N * q > 2
    np.testing.assert_allclose(var[big], (N * q * (1 - q))[big], rtol=0.25)
    one = np.zeros(N)
    one[17] = 1.0
    np.testing.assert_array_equal(O.resample_multinomial(one, rng.random(N)), np.full(N, 17))
    np.testing.assert_array_equal(O.resample_multinomial(np.zeros(N), rng.random(N)), np.arange(N))


def test_multinomial_uniforms_are_the_second_draw_of_each_offspring_block():
    seed, stage, N = 77, 5, 9
    U = O.multinomial_uniforms(seed, stage, N)
    for i in range(N):
        out = O.philox4x32_10([0, i, O.stage_move(stage, 0), O.TAG_RESAMPLE],
                              [seed & 0xFFFFFFFF, seed >> 32])
        r = (int(out[3]) << 32) | int(out[2])
        assert U[i] == (r >> 11) * 2.0 ** -53


# ----------------------------------------------------------------------------------------------
# Moves (Algorithm 1)
# ----------------------------------------------------------------------------------------------
def test_upm_move_changes_one_block_with_the_drawn_indices():
    wl = small_glm("gaussian", n=300, p=3, N=16, m=20, G=4, seed=2)
    prob = O.Problem("gaussian", wl.X, wl.y, wl.prior_mean, wl.prior_var, sigma=wl.sigma)
    prob.set_centre(np.zeros(3))
    th, us = O.init_particles(5, wl.N, 3, wl.m, wl.n, wl.prior_mean, wl.prior_var)
    old = us.copy()
    acc = O.upm_move(prob, wl.m, wl.G, 5, 3, 1, 0.6, th, us)
    assert acc.all()  # exact control variates: r = 1 (Eq. acc_prop_u)
    sm = O.stage_move(3, 1)
    for i in range(wl.N):
        g = O.index(O.r64(5, O.TAG_UPM_BLOCK, sm, i, 0), wl.G)
        lo, hi = (g * wl.m) // wl.G, ((g + 1) * wl.m) // wl.G
        np.testing.assert_array_equal(us[i, :lo], old[i, :lo])
        np.testing.assert_array_equal(us[i, hi:], old[i, hi:])
        want = [O.index(O.r64(5, O.TAG_UPM_IDX, sm, i, j), wl.n) for j in range(hi - lo)]
        np.testing.assert_array_equal(us[i, lo:hi], want)


def test_upm_move_acceptance_matches_mh_ratio():
    wl = small_glm("logistic", n=500, p=3, N=32, m=10, G=2, seed=4)
    prob = O.Problem("logistic", wl.X, wl.y, wl.prior_mean, wl.prior_var)
    prob.set_centre(wl.theta_true)
    th, us = O.init_particles(9, wl.N, 3, wl.m, wl.n, wl.prior_mean, wl.prior_var * 0.01)
    th += wl.theta_true
    before = O.loglik_batch(prob, wl.m, wl.G, th, us, grad=False)
    us2 = us.copy()
    a = 0.9
    acc = O.upm_move(prob, wl.m, wl.G, 9, 1, 0, a, th, us2)
    after = O.loglik_batch(prob, wl.m, wl.G, th, us2, grad=False)
    sm = O.stage_move(1, 0)
    n_acc = 0
    for i in range(wl.N):
        if not acc[i]:
            np.testing.assert_array_equal(us2[i], us[i])
            continue
        n_acc += 1
        logr = (a * after["ell"][i] - 0.5 * a * a * after["sigma2"][i]) - (
            a * before["ell"][i] - 0.5 * a * a * before["sigma2"][i])
        assert math.log(O.uniform(O.r64(9, O.TAG_MH_U, sm, i, 0))) < logr + 1e-9
    assert 0 < n_acc < wl.N


def _conjugate(n=200, p=3, sigma=0.8, tau2=4.0, seed=3):
    wl = small_glm("gaussian", n=n, p=p, N=1, m=1, G=1, seed=seed, sigma=sigma,
                   prior_var=tau2)
    prob = O.Problem("gaussian", wl.X, wl.y, wl.prior_mean, wl.prior_var, sigma=sigma)
    X, y = wl.X, wl.y
    S = np.linalg.inv(X.T @ X / sigma ** 2 + np.eye(p) / tau2)
    mu = S @ X.T @ y / sigma ** 2
    logml = stats.multivariate_normal(mean=np.zeros(n),
                                      cov=sigma ** 2 * np.eye(n) + tau2 * X @ X.T).logpdf(y)
    return prob, mu, S, float(logml)


def test_hmc_small_step_accepts_everything_and_large_step_is_valid():
    prob, mu, S, _ = _conjugate()
    prob.set_centre(mu)
    N, m = 64, 10
    th, us = O.init_particles(4, N, prob.p, m, prob.n, prob.prior_mean, prob.prior_var)
    th = mu + (th / np.sqrt(prob.prior_var)) @ np.linalg.cholesky(S).T
    Lc = np.linalg.cholesky(S)
    acc = O.hmc_move(prob, m, 2, 4, 1, 0, 1.0, 1e-3, 5, S, Lc, th.copy(), us)
    assert acc.all()
    acc = O.hmc_move(prob, m, 2, 4, 1, 1, 1.0, 0.9, 5, S, Lc, th.copy(), us)
    assert 0.5 < acc.mean() <= 1.0


def test_hmc_leaves_exact_posterior_invariant():
    """Conjugate Gaussian model at a=1: start from exact posterior draws, apply HMC moves with
    the posterior covariance as Sigma; the draws stay distributed as N(mu, S)."""
    prob, mu, S, _ = _conjugate()
    prob.set_centre(mu)
    N, m = 2000, 5
    rng = np.random.default_rng(0)
    Lc = np.linalg.cholesky(S)
    th = mu + rng.standard_normal((N, prob.p)) @ Lc.T
    us = rng.integers(0, prob.n, size=(N, m)).astype(np.int64)
    for r in range(3):
        O.hmc_move(prob, m, 1, 21, 1, r, 1.0, 0.7, 8, S, Lc, th, us)
    z = np.linalg.solve(Lc, (th - mu).T).T  # whitened: should be N(0, I)
    assert np.all(np.abs(z.mean(axis=0)) < 4 / math.sqrt(N))
    assert np.all(np.abs(z.var(axis=0) - 1.0) < 5 * math.sqrt(2.0 / N))


def _conjugate_tempered_log_z(prob, a):
    """log of the integral of p(y | theta)^a p(theta) for the conjugate Gaussian model (prior
    N(0, tau2 I)), in closed form: with Lam = a X'X / s^2 + I / tau2 and b = a X'y / s^2,
    -(a n / 2) log 2 pi s^2 - log det(tau2 Lam) / 2 + b' Lam^-1 b / 2 - a y'y / (2 s^2)."""
    X, y, s2, tau2 = prob.X, prob.y, prob.sigma ** 2, prob.prior_var[0]
    n, p = X.shape
    lam = a * X.T @ X / s2 + np.eye(p) / tau2
    b = a * X.T @ y / s2
    return (-0.5 * a * n * math.log(2 * math.pi * s2) - 0.5 * np.linalg.slogdet(tau2 * lam)[1]
            + 0.5 * b @ np.linalg.solve(lam, b) - a * (y @ y) / (2 * s2))


def test_smc_recovers_conjugate_posterior_and_log_marginal():
    """Averaged over 8 seeded runs (the paper repeats each run 10 times for its standard errors):
    single-run log-ML sd is about 0.13 at N=1024, so the mean is held to 0.15. The running sum of
    the stage increments (Sec. 3.5) is also held, stage by stage, to the closed-form log evidence
    of the tempered posterior at that stage's temperature."""
    prob, mu, S, logml = _conjugate()
    prob.set_centre(mu)
    assert _conjugate_tempered_log_z(prob, 1.0) == pytest.approx(logml, abs=1e-9)
    assert _conjugate_tempered_log_z(prob, 0.0) == pytest.approx(0.0, abs=1e-12)
    errs, means, path_errs = [], [], []
    for seed in range(1, 9):
        cfg = O.SMCConfig(N=1024, m=8, G=2, L=8, R=3, seed=seed, tau=0.5)
        st = O.smc_run(prob, cfg)
        assert st.a == 1.0 and st.stage >= 2
        errs.append(st.log_z - logml)
        means.append(st.thetas.mean(axis=0))
        running = np.cumsum([h["log_z_inc"] for h in st.history])
        path_errs.append([z - _conjugate_tempered_log_z(prob, h["a"])
                          for z, h in zip(running, st.history)])
    sd = np.sqrt(np.diag(S))
    assert np.all(np.abs(np.mean(means, axis=0) - mu) < 0.05 * sd)
    assert abs(np.mean(errs)) < 0.15
    assert np.max(np.abs(errs)) < 0.6
    k = min(len(e) for e in path_errs)
    assert np.all(np.abs(np.mean([e[:k] for e in path_errs], axis=0)) < 0.1)
    assert max(np.max(np.abs(e)) for e in path_errs) < 0.5


@pytest.mark.parametrize("fam", ["logistic", "poisson", "probit"])
def test_first_order_estimator_unbiased_and_its_gradient(fam):
    """First-order control variates (q_k = l_k(tb) + grad l_k(tb)'delta): averaging l_hat over all
    n^m index tuples gives l(theta) exactly, the printed sigma2_hat has expectation
    (m-1)/m Var(l_hat), l_hat = A at the centre, and the force is the gradient of the target."""
    n, m = 5, 3
    prob = tiny_problem(fam, n=n, p=2, seed=11)
    prob.cv_order = 1
    theta = prob.theta_bar + np.array([0.4, -0.7])
    us = np.array([[a, b, c] for a in range(n) for b in range(n) for c in range(n)],
                  dtype=np.int64)
    thetas = np.repeat(theta[None, :], us.shape[0], axis=0)
    out = O.loglik_batch(prob, m, 1, thetas, us, a=1.0, grad=False)
    exact = scipy_loglik(fam, prob.X, prob.y, theta, prob.sigma)
    assert out["ell"].mean() == pytest.approx(exact, rel=1e-12)
    assert out["sigma2"].mean() == pytest.approx((m - 1) / m * out["ell"].var(), rel=1e-10)
    # first and second order differ (the check is not vacuous)
    prob.cv_order = 2
    out2 = O.loglik_batch(prob, m, 1, thetas, us, a=1.0, grad=False)
    assert np.max(np.abs(out2["ell"] - out["ell"])) > 1e-6
    prob.cv_order = 1
    o = O.loglik_batch(prob, m, 1, prob.theta_bar[None, :], us[:1], a=1.0, grad=False)
    assert o["ell"][0] == pytest.approx(prob.A, rel=1e-14)
    prob2 = tiny_problem(fam, n=40, p=3, seed=4)
    prob2.cv_order = 1
    rng = np.random.default_rng(8)
    mm, a = 12, 0.7
    u = rng.integers(0, prob2.n, size=(1, mm)).astype(np.int64)
    th = prob2.theta_bar + 0.5 * rng.standard_normal(prob2.p)

    def target(t):
        r = O.loglik_batch(prob2, mm, 3, t[None, :], u, a=a, grad=False)
        return (a * r["ell"][0] - 0.5 * a * a * r["sigma2"][0]
                + scipy_log_prior(t, prob2.prior_mean, prob2.prior_var))

    g = O.loglik_batch(prob2, mm, 3, th[None, :], u, a=a)["grad"][0]
    h = 1e-6
    for c in range(prob2.p):
        e = np.zeros(prob2.p)
        e[c] = h
        fd = (target(th + e) - target(th - e)) / (2 * h)
        assert g[c] == pytest.approx(fd, rel=1e-6, abs=1e-6)


@pytest.mark.parametrize("mode", [1, 2])
def test_recentred_smc_gaussian_matches_fixed_centre(mode):
    """Algorithm 2 (d) moves theta_bar to the reweighted particle mean every stage. For the
    Gaussian family the second-order expansion is exact, so l_hat does not depend on the centre:
    a run started from a poor centre and re-centred every stage must follow the fixed-centre run
    to rounding. A wrong A, B or C at the new centre shifts l_hat and the whole trajectory."""
    prob, mu, S, logml = _conjugate()
    prob.set_centre(np.zeros(prob.p))
    cfg = O.SMCConfig(N=256, m=8, G=2, L=6, R=2, seed=5, tau=0.5)
    st0 = O.smc_run(prob, cfg)
    prob.set_centre(np.zeros(prob.p))
    cfg_r = O.SMCConfig(N=256, m=8, G=2, L=6, R=2, seed=5, tau=0.5, recentre=mode)
    st1 = O.smc_run(prob, cfg_r)
    assert st1.stage == st0.stage
    assert st1.log_z == pytest.approx(st0.log_z, abs=1e-8)
    np.testing.assert_allclose(st1.thetas, st0.thetas, rtol=1e-8, atol=1e-10)
    # the centre moved to the last stage's reweighted mean, near the posterior mean
    sd = np.sqrt(np.diag(S))
    assert np.all(np.abs(prob.theta_bar - mu) < 0.5 * sd)
    assert abs(st1.log_z - logml) < 0.6


def _logistic_quadrature(seed=2, n=400):
    """A two-parameter logistic posterior and its log marginal likelihood by tensor-grid
    quadrature (independent of the oracle: scipy's Bernoulli log-pmf on a 301 x 301 grid)."""
    rng = np.random.default_rng(seed)
    X = np.column_stack([np.ones(n), rng.standard_normal(n)])
    y = (rng.random(n) < special.expit(X @ np.array([0.6, -1.2]))).astype(float)
    var = np.full(2, 4.0)
    prob = O.Problem("logistic", X, y, np.zeros(2), var)
    g = [np.linspace(-1.5, 2.5, 301), np.linspace(-3.5, 0.5, 301)]
    T0, T1 = np.meshgrid(g[0], g[1], indexing="ij")
    eta = X[:, 0, None, None] * T0[None] + X[:, 1, None, None] * T1[None]
    lp = (stats.bernoulli.logpmf(y[:, None, None], special.expit(eta)).sum(axis=0)
          + stats.norm.logpdf(T0, 0, 2.0) + stats.norm.logpdf(T1, 0, 2.0))
    dA = (g[0][1] - g[0][0]) * (g[1][1] - g[1][0])
    logml = float(special.logsumexp(lp) + math.log(dA))
    w = np.exp(lp - lp.max())
    w /= w.sum()
    mean = np.array([(w * T0).sum(), (w * T1).sum()])
    sd = np.sqrt(np.array([(w * (T0 - mean[0]) ** 2).sum(), (w * (T1 - mean[1]) ** 2).sum()]))
    return prob, mean, sd, logml


@pytest.mark.parametrize("order,mode", [(2, 1), (1, 1), (2, 2)])
def test_recentred_logistic_smc_against_quadrature(order, mode):
    """Subsampled SMC re-centred every stage (Algorithm 2 (d)), from a centre at the prior mean,
    with second- or first-order control variates (Sec. 4's Experiment 4): the log marginal
    likelihood and the posterior mean agree with grid quadrature. Four seeded runs are averaged."""
    prob, mean, sd, logml = _logistic_quadrature()
    prob.cv_order = order
    errs, means = [], []
    for seed in range(1, 5):
        prob.set_centre(np.zeros(2))
        cfg = O.SMCConfig(N=1024, m=40, G=4, L=8, R=3, seed=seed, tau=0.5, recentre=mode)
        st = O.smc_run(prob, cfg)
        assert st.a == 1.0
        errs.append(st.log_z - logml)
        means.append(st.thetas.mean(axis=0))
        assert np.all(np.abs(prob.theta_bar - mean) < 0.5 * sd)
    assert np.all(np.abs(np.mean(means, axis=0) - mean) < 0.1 * sd)
    assert abs(np.mean(errs)) < 0.2


def test_paper_settings_recover_conjugate_posterior_and_log_marginal():
    """The paper's own settings together: ESS target 0.8N by the grid rule, multinomial
    resampling, control variates re-centred every stage (Algorithm 2 as printed). Averaged over
    six seeded runs on the conjugate Gaussian model, against the closed forms."""
    prob, mu, S, logml = _conjugate()
    errs, means = [], []
    for seed in range(1, 7):
        prob.set_centre(np.zeros(prob.p))
        cfg = O.SMCConfig(N=1024, m=8, G=2, L=8, R=3, seed=seed, tau=0.8, recentre=1,
                          resampling="multinomial", grid_points=512, grid_decades=16.0)
        st = O.smc_run(prob, cfg)
        assert st.a == 1.0
        assert all(abs(h["ess"] - 0.8 * cfg.N) < 0.05 * cfg.N for h in st.history[:-1])
        errs.append(st.log_z - logml)
        means.append(st.thetas.mean(axis=0))
    sd = np.sqrt(np.diag(S))
    assert np.all(np.abs(np.mean(means, axis=0) - mu) < 0.05 * sd)
    assert abs(np.mean(errs)) < 0.15


def test_student_t_newton_reaches_the_mode_from_a_non_concave_start():
    """Student-t regression (Sec. 4.3) far from the mode has an indefinite Hessian; the damped
    Newton steps still end at a stationary point of the log posterior that is a maximum (the
    gradient rebuilt from scipy's log-density by finite differences, the Hessian negative
    definite), and the plain posterior mode found by scipy's optimiser agrees."""
    from scipy import optimize
    rng = np.random.default_rng(21)
    n, p = 400, 3
    X = np.column_stack([np.ones(n), rng.standard_normal((n, p - 1))])
    theta = np.array([6.0, -4.0, 5.0])  # residuals of ~8 at the prior mean: l'' > 0 there
    y = X @ theta + 0.8 * rng.standard_t(5.0, size=n)
    prob = O.Problem("student_t", X, y, np.zeros(p), np.full(p, 10.0), sigma=0.8, dof=5.0)
    _, _, C0 = O.cv_moments("student_t", X, y, np.zeros(p), 0.8, 5.0)
    assert np.max(np.linalg.eigvalsh(-C0 + np.eye(p) / 10.0)) > 0  # some curvature is wrong-signed
    assert np.min(np.linalg.eigvalsh(-C0 + np.eye(p) / 10.0)) < 0
    mode = O.newton_map(prob)

    def neg_logpost(t):
        return -(scipy_loglik("student_t", X, y, t, 0.8)
                 + scipy_log_prior(t, prob.prior_mean, prob.prior_var))

    h = 1e-6
    g = np.array([(neg_logpost(mode + h * e) - neg_logpost(mode - h * e)) / (2 * h)
                  for e in np.eye(p)])
    assert np.max(np.abs(g)) < 1e-4
    _, _, C = O.cv_moments("student_t", X, y, mode, 0.8, 5.0)
    assert np.max(np.linalg.eigvalsh(C - np.eye(p) / 10.0)) < 0
    ref = optimize.minimize(neg_logpost, mode + 0.3, method="BFGS", options={"gtol": 1e-9})
    np.testing.assert_allclose(mode, ref.x, atol=1e-5)



def test_componentwise_correlation_and_the_adaptive_rule():
    """The adaptive number of moves (Sec. 3.4): correlations against numpy's corrcoef, and the
    rule reads the ceil(q p)-th smallest of them."""
    rng = np.random.default_rng(30)
    th0 = rng.standard_normal((500, 6))
    th = 0.3 * th0 + rng.standard_normal((500, 6)) * np.linspace(0.1, 3.0, 6)
    rho = O.componentwise_correlation(th0, th)
    for c in range(6):
        assert rho[c] == pytest.approx(np.corrcoef(th0[:, c], th[:, c])[0, 1], rel=1e-12)
    srt = np.sort(rho)
    # q = 0.9 with p = 6: the 6th smallest (the largest); q = 0.5: the 3rd smallest
    assert O.decorrelated(th0, th, srt[5], 0.9) and not O.decorrelated(th0, th, srt[4], 0.9)
    assert O.decorrelated(th0, th, srt[2], 0.5) and not O.decorrelated(th0, th, srt[1], 0.5)
    flat = th.copy()
    flat[:, 0] = 1.0  # no spread: counts as still correlated
    assert O.componentwise_correlation(th0, flat)[0] == 1.0


def test_adaptive_moves_recover_conjugate_posterior():
    """Runs whose move counts follow the adaptive rule recover the conjugate posterior and log
    marginal likelihood (seed-averaged); a lower threshold needs at least as many moves."""
    prob, mu, S, logml = _conjugate()
    prob.set_centre(mu)
    errs, means, Rs = [], [], {0.5: [], 0.05: []}
    for seed in range(1, 7):
        for rho_max in (0.5, 0.05):
            cfg = O.SMCConfig(N=1024, m=8, G=2, L=8, R=1, seed=seed, tau=0.5,
                              adaptive=(40, rho_max, 0.9))
            st = O.smc_run(prob, cfg)
            Rs[rho_max] += [h["R"] for h in st.history]
            if rho_max == 0.05:
                errs.append(st.log_z - logml)
                means.append(st.thetas.mean(axis=0))
    assert np.mean(Rs[0.05]) > np.mean(Rs[0.5]) >= 1.0
    assert 1 <= min(Rs[0.05]) and max(Rs[0.05]) <= 40
    sd = np.sqrt(np.diag(S))
    assert np.all(np.abs(np.mean(means, axis=0) - mu) < 0.05 * sd)
    assert abs(np.mean(errs)) < 0.15


def test_rw_move_proposal_and_invariance():
    """Random-walk Metropolis (Sec. 4.2's RW kernel): at a tiny step every proposal
    theta + eps Lc z is accepted (z rebuilt from the momentum stream's normals); started at exact
    conjugate posterior draws with Sigma the posterior covariance, the moves keep them N(mu, S)."""
    prob, mu, S, _ = _conjugate()
    prob.set_centre(mu)
    Lc = np.linalg.cholesky(S)
    N, m, seed, stage = 64, 5, 13, 2
    rng = np.random.default_rng(1)
    th = mu + rng.standard_normal((N, prob.p)) @ Lc.T
    us = rng.integers(0, prob.n, size=(N, m)).astype(np.int64)
    th1 = th.copy()
    acc = O.rw_move(prob, m, 1, seed, stage, 0, 1.0, 1e-6, Lc, th1, us)
    assert acc.all()
    for i in range(N):
        z = np.array([O.normal(seed, O.TAG_MOMENTUM, O.stage_move(stage, 0), i, c)
                      for c in range(prob.p)])
        np.testing.assert_allclose(th1[i], th[i] + 1e-6 * Lc @ z, rtol=0, atol=1e-15)
    N = 4000
    th = mu + rng.standard_normal((N, prob.p)) @ Lc.T
    us = rng.integers(0, prob.n, size=(N, m)).astype(np.int64)
    rates = []
    for r in range(6):
        rates.append(O.rw_move(prob, m, 1, seed, stage, r, 1.0, 2.38 / math.sqrt(prob.p), Lc, th,
                               us).mean())
    assert 0.15 < np.mean(rates) < 0.6
    z = np.linalg.solve(Lc, (th - mu).T).T
    assert np.all(np.abs(z.mean(axis=0)) < 4 / math.sqrt(N))
    assert np.all(np.abs(z.var(axis=0) - 1.0) < 5 * math.sqrt(2.0 / N))


def test_rw_smc_recovers_conjugate_posterior():
    prob, mu, S, logml = _conjugate()
    prob.set_centre(mu)
    errs, means = [], []
    for seed in range(1, 7):
        cfg = O.SMCConfig(N=1024, m=8, G=2, L=1, R=8, seed=seed, tau=0.5, theta_move="rw",
                          eps0=1.0)
        st = O.smc_run(prob, cfg)
        errs.append(st.log_z - logml)
        means.append(st.thetas.mean(axis=0))
    sd = np.sqrt(np.diag(S))
    assert np.all(np.abs(np.mean(means, axis=0) - mu) < 0.05 * sd)
    assert abs(np.mean(errs)) < 0.15


def _prior_only_case(seed=17, N=40):
    prob = tiny_problem("logistic", n=30, p=3, seed=6)
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3, 3))
    Sigma = A @ A.T + 0.5 * np.eye(3)
    Lc = np.linalg.cholesky(Sigma)
    th = prob.prior_mean + rng.standard_normal((N, 3)) * 2.0
    us = rng.integers(0, prob.n, size=(N, 4)).astype(np.int64)
    return prob, Sigma, Lc, th, us


def _log_prior(t, prob):
    return float(np.sum(-0.5 * (t - prob.prior_mean) ** 2 / prob.prior_var
                        - 0.5 * np.log(2 * np.pi * prob.prior_var)))


@pytest.mark.parametrize("jitter", [0.0, 0.3])
def test_hmc_move_at_zero_temperature_matches_a_direct_leapfrog(jitter):
    """At a = 0 the target is the prior alone, so the whole HMC move can be rebuilt in numpy from
    its definition: momentum rho = Lc^-T z (z the momentum stream's normals), the particle's step
    eps (1 - j + 2 j U) with U its theta-MH block's second word, L leapfrog steps under the
    prior's force, H = -log p(theta) + rho' Sigma rho / 2, accept when log U0 < H0 - H1 (U0 the
    first word). Accept decisions and end points agree with the oracle's move."""
    prob, Sigma, Lc, th, us = _prior_only_case()
    seed, stage, move, eps, L = 23, 4, 1, 1.2, 7
    sm = O.stage_move(stage, move)
    th_o = th.copy()
    acc = O.hmc_move(prob, 4, 2, seed, stage, move, 0.0, eps, L, Sigma, Lc, th_o, us,
                     jitter=jitter)
    for i in range(th.shape[0]):
        z = np.array([O.normal(seed, O.TAG_MOMENTUM, sm, i, c) for c in range(3)])
        rho = np.linalg.solve(Lc.T, z)
        e = eps
        if jitter > 0:
            e = eps * (1 - jitter + 2 * jitter * O.uniform(O.r64(seed, O.TAG_MH_THETA, sm, i, 1)))
        t = th[i].copy()
        force = lambda x: -(x - prob.prior_mean) / prob.prior_var
        H0 = -_log_prior(t, prob) + 0.5 * rho @ Sigma @ rho
        for _ in range(L):
            rho = rho + 0.5 * e * force(t)
            t = t + e * (Sigma @ rho)
            rho = rho + 0.5 * e * force(t)
        H1 = -_log_prior(t, prob) + 0.5 * rho @ Sigma @ rho
        ok = math.log(O.uniform(O.r64(seed, O.TAG_MH_THETA, sm, i, 0))) < H0 - H1
        assert bool(acc[i]) == ok, i
        np.testing.assert_allclose(th_o[i], t if ok else th[i], rtol=1e-12, atol=1e-12)
    assert 0 < acc.sum() < th.shape[0]  # both outcomes are exercised at this step


def test_rw_move_at_zero_temperature_matches_its_definition():
    prob, Sigma, Lc, th, us = _prior_only_case(seed=3)
    seed, stage, move, eps = 31, 2, 0, 1.3
    sm = O.stage_move(stage, move)
    th_o = th.copy()
    acc = O.rw_move(prob, 4, 2, seed, stage, move, 0.0, eps, Lc, th_o, us)
    for i in range(th.shape[0]):
        z = np.array([O.normal(seed, O.TAG_MOMENTUM, sm, i, c) for c in range(3)])
        t = th[i] + eps * Lc @ z
        ok = (math.log(O.uniform(O.r64(seed, O.TAG_MH_THETA, sm, i, 0)))
              < _log_prior(t, prob) - _log_prior(th[i], prob))
        assert bool(acc[i]) == ok, i
        np.testing.assert_allclose(th_o[i], t if ok else th[i], rtol=1e-12, atol=1e-12)
    assert 0 < acc.sum() < th.shape[0]


def test_initial_particles_follow_the_prior_and_p_of_u():
    """Algorithm 2 step 1: theta ~ N(prior mean, diag(prior var)) and u iid uniform on {0..n-1}."""
    N, p, m, n = 20000, 3, 6, 17
    mu, var = np.array([0.5, -2.0, 0.0]), np.array([0.25, 4.0, 10.0])
    th, us = O.init_particles(5, N, p, m, n, mu, var)
    se = np.sqrt(var / N)
    assert np.all(np.abs(th.mean(axis=0) - mu) < 5 * se)
    assert np.all(np.abs(th.var(axis=0) / var - 1.0) < 5 * math.sqrt(2.0 / N))
    assert np.abs(np.corrcoef(th.T)[np.triu_indices(p, 1)]).max() < 5 / math.sqrt(N)
    counts = np.bincount(us.ravel(), minlength=n)
    assert us.min() >= 0 and us.max() < n
    assert stats.chisquare(counts).pvalue > 1e-4
    # different particles and different slots draw independently
    assert abs(np.corrcoef(us[:, 0], us[:, 1])[0, 1]) < 5 / math.sqrt(N)


def test_singular_particle_covariance_gets_the_documented_jitter():
    """A cloud on a line has a singular covariance: the diagonal receives 1e-10 tr/p, times 10
    per retry, cumulatively, until the Cholesky factorisation succeeds."""
    rng = np.random.default_rng(4)
    N, p = 200, 3
    t = rng.standard_normal(N)
    th = np.outer(t, [1.0, -2.0, 0.5]) + np.array([0.3, 0.1, -0.2])
    W = np.full(N, 1.0 / N)
    mean, S, Lc, rc = O.moments(W, th)
    S0 = np.cov(th.T, aweights=W, ddof=0)
    assert rc >= 1
    jit0 = 1e-10 * np.trace(S0) / p
    added = jit0 * sum(10.0 ** k for k in range(rc))
    np.testing.assert_allclose(S - S0, added * np.eye(p), rtol=1e-6, atol=1e-15)
    np.testing.assert_allclose(Lc @ Lc.T, S, rtol=1e-9, atol=1e-12 * np.abs(S).max())


def test_smc_log_marginal_on_the_plain_logistic_workload_against_importance_sampling():
    """The plain FP64 workload (logistic, n = 10,000, p = 5): a reference log marginal likelihood
    by importance sampling with a multivariate-t (5 degrees of freedom) proposal at the mode with
    the Laplace covariance (tests/logml_reference.py: numpy/scipy only; 40,000 draws, relative
    standard error of the estimate of p(y) about 0.2%). The oracle's SMC at N = 1024 recovers it:
    mean error over eight seeded runs within 0.15 (about 2.5 standard errors of that mean)."""
    from logml_reference import importance_reference
    from smc_workloads import logistic_1e4
    wl = logistic_1e4()
    prob = O.Problem("logistic", wl.X, wl.y, wl.prior_mean, wl.prior_var)
    mode = O.newton_map(prob)
    prob.set_centre(mode)
    ref_d = importance_reference(wl.X, wl.y, wl.prior_var)
    np.testing.assert_allclose(ref_d["mode"], mode, rtol=1e-9, atol=1e-10)
    assert ref_d["rel_se"] < 0.01
    ref = ref_d["log_ml"]
    errs = []
    for seed in range(1, 9):
        st = O.smc_run(prob, O.SMCConfig(N=1024, m=100, G=10, L=10, R=5, seed=seed, tau=0.5))
        errs.append(st.log_z - ref)
    assert abs(np.mean(errs)) < 0.15, errs
    assert np.max(np.abs(errs)) < 0.7, errs


def test_hmc_at_zero_temperature_keeps_prior_draws_prior_distributed():
    """a = 0: the extended target is the prior (times p(u)); moves started from prior draws leave
    the cloud distributed as the prior (moments within Monte Carlo error)."""
    prob = tiny_problem("poisson", n=40, p=3, seed=2)
    N, m = 6000, 5
    mu, var = prob.prior_mean, prob.prior_var
    th, us = O.init_particles(8, N, 3, m, prob.n, mu, var)
    S = np.diag(var)
    Lc = np.linalg.cholesky(S)
    for r in range(3):
        O.upm_move(prob, m, 1, 8, 1, r, 0.0, th, us)
        O.hmc_move(prob, m, 1, 8, 1, r, 0.0, 0.8, 6, S, Lc, th, us)
    z = (th - mu) / np.sqrt(var)
    assert np.all(np.abs(z.mean(axis=0)) < 5 / math.sqrt(N))
    assert np.all(np.abs(z.var(axis=0) - 1.0) < 5 * math.sqrt(2.0 / N))


def test_move_margins_are_the_decisions_distance_from_the_threshold():
    """The optional margin record of the oracle's moves (test support): for the u update the margin
    equals a (l_hat* - l_hat) - a^2/2 (sigma2* - sigma2) - log U rebuilt here from the oracle's
    estimator at the proposed indices (block and indices redrawn from the raw Philox streams);
    for both moves the margin is positive exactly where the move was accepted."""
    prob = tiny_problem("logistic", n=60, p=3, seed=5)
    N, m, G, seed, stage, a = 40, 9, 3, 21, 4, 0.7
    th, us = O.init_particles(seed, N, 3, m, prob.n, prob.prior_mean, prob.prior_var)
    th = prob.theta_bar + 0.3 * (th - prob.prior_mean) / np.sqrt(prob.prior_var)
    us0 = us.copy()
    mu = np.zeros(N)
    acc = O.upm_move(prob, m, G, seed, stage, 0, a, th, us, margins=mu)
    assert np.array_equal(mu > 0, acc.astype(bool))
    sm = O.stage_move(stage, 0)
    ustar = us0.copy()
    for i in range(N):
        g = O.index(O.r64(seed, O.TAG_UPM_BLOCK, sm, i, 0), G)
        j0, j1 = (g * m) // G, ((g + 1) * m) // G
        for j in range(j0, j1):
            ustar[i, j] = O.index(O.r64(seed, O.TAG_UPM_IDX, sm, i, j - j0), prob.n)
    r0 = O.loglik_batch(prob, m, G, th, us0, grad=False)
    r1 = O.loglik_batch(prob, m, G, th, ustar, grad=False)
    logU = np.log([O.uniform(O.r64(seed, O.TAG_MH_U, sm, i, 0)) for i in range(N)])
    want = a * (r1["ell"] - r0["ell"]) - 0.5 * a * a * (r1["sigma2"] - r0["sigma2"]) - logU
    np.testing.assert_allclose(mu, want, rtol=1e-12, atol=1e-12)
    S = np.diag([0.05, 0.02, 0.02])
    mh = np.zeros(N)
    acc = O.hmc_move(prob, m, G, seed, stage, 1, a, 2.5, 4, S, np.linalg.cholesky(S), th, us,
                     margins=mh)
    assert np.array_equal(mh > 0, acc.astype(bool)) and 0 < acc.sum() < N


@pytest.mark.parametrize("fam", ["logistic", "probit", "poisson", "gaussian", "student_t"])
def test_hmc_energy_error_is_second_order_in_the_step(fam):
    """Leapfrog is a second-order integrator, so over a fixed trajectory time the change of the
    Hamiltonian H = -log target + rho' Sigma rho / 2 shrinks by 4 each time the step is halved,
    provided the force is the exact gradient of the log target that H uses (here a l_hat -
    a^2 sigma2_hat / 2 + log p, at a = 0.8 so that the sigma2_hat term counts). A force that
    missed a term, a wrong sign, the inverse mass matrix in place of Sigma, or a first-order
    update would leave a ratio near 1 or 2. H1 - H0 is read from the move's MH margin
    (H0 - H1 - log U) with log U rebuilt from the raw Philox stream; the step is fixed (no
    jitter) and the same momentum is drawn at every step size."""
    prob = tiny_problem(fam, n=200, p=3, seed=7)
    N, m, G, seed, stage, a = 48, 40, 4, 13, 3, 0.8
    th, us = O.init_particles(seed, N, 3, m, prob.n, prob.prior_mean, prob.prior_var)
    th = prob.theta_bar + 0.15 * (th - prob.prior_mean) / np.sqrt(prob.prior_var)
    S = np.diag([0.05, 0.03, 0.03])
    Lc = np.linalg.cholesky(S)
    sm = O.stage_move(stage, 0)
    logU = np.log([O.uniform(O.r64(seed, O.TAG_MH_THETA, sm, i, 0)) for i in range(N)])
    dH = []
    for eps, L in [(0.04, 16), (0.02, 32), (0.01, 64)]:  # trajectory time 0.64 each
        margin = np.zeros(N)
        O.hmc_move(prob, m, G, seed, stage, 0, a, eps, L, S, Lc, th.copy(), us, jitter=-1.0,
                   margins=margin)
        dH.append(-(margin + logU))
    assert np.abs(dH[-1]).max() > 1e-6  # far above rounding: the ratios below measure the method
    for big, small in zip(dH[:-1], dH[1:]):
        assert 3.9 < np.abs(big).sum() / np.abs(small).sum() < 4.1
        assert 3.9 < np.median(big / small) < 4.1


@pytest.mark.parametrize("fam", ["logistic", "probit", "poisson", "gaussian", "student_t"])
def test_leapfrog_is_reversible_and_volume_preserving(fam):
    """The two properties that make the HMC move's acceptance ratio (Algorithm 1 step 2) the
    Hamiltonian difference alone, checked on the move's own leapfrog routine: L steps from
    (theta, rho), then L steps from the end point with the momentum negated, return to
    (theta, -rho) up to rounding (time reversibility); and the Jacobian of the map
    (theta, rho) -> (theta_L, rho_L), by central differences, has determinant 1 (volume
    preservation). A non-symmetric step (a full first kick, a missing last half kick) fails the
    first."""
    prob = tiny_problem(fam, n=200, p=3, seed=7)
    m, G, a, eps, L = 40, 4, 0.8, 0.05, 12
    _, us = O.init_particles(17, 1, 3, m, prob.n, prob.prior_mean, prob.prior_var)
    rng = np.random.default_rng(5)
    theta = prob.theta_bar + 0.1 * rng.standard_normal(3)
    S = np.array([[0.05, 0.01, 0.0], [0.01, 0.03, 0.005], [0.0, 0.005, 0.03]])
    rho = np.linalg.solve(np.linalg.cholesky(S).T, rng.standard_normal(3))  # N(0, S^-1)
    th1, r1, _ = O.leapfrog(prob, m, G, us[0], a, eps, L, S, theta, rho)
    assert np.linalg.norm(th1 - theta) > 0.02  # the trajectory went somewhere
    th2, r2, _ = O.leapfrog(prob, m, G, us[0], a, eps, L, S, th1, -r1)
    np.testing.assert_allclose(th2, theta, rtol=0, atol=1e-11)
    np.testing.assert_allclose(-r2, rho, rtol=0, atol=1e-10 * np.abs(rho).max())

    def flow(z):
        t, r, _ = O.leapfrog(prob, m, G, us[0], a, eps, L, S, z[:3], z[3:])
        return np.concatenate([t, r])

    z0, h = np.concatenate([theta, rho]), 1e-6
    J = np.column_stack([(flow(z0 + h * e) - flow(z0 - h * e)) / (2 * h) for e in np.eye(6)])
    assert abs(np.linalg.det(J) - 1.0) < 1e-6


@pytest.mark.parametrize("fam,scale", [("logistic", 1.5), ("probit", 1.0), ("poisson", 0.5),
                                       ("student_t", 0.4)])
def test_upm_move_leaves_the_extended_target_of_u_invariant(fam, scale):
    """At fixed theta the u update (Algorithm 1 step 1, Eq. acc_prop_u) must leave the u-marginal
    of the extended target invariant: pi(u) proportional to exp(a l_hat(u) - a^2 sigma2_hat(u)/2)
    p(u), with p(u) uniform over index tuples (Eq. extended_target_at_sequence_p). With n = 6 and
    m = 2 there are 36 tuples, so pi is computed exactly from the (separately pinned) estimator;
    40,000 particles start from exact pi draws, take ten moves, and their tuple histogram must
    still fit pi (chi-square, expected counts under 5 pooled). theta sits far enough from the
    centre that the sigma2_hat term moves pi by a total variation of 0.1-0.25 (a flipped sign),
    and a = 0.7 keeps a and a^2 apart."""
    import itertools
    prob = tiny_problem(fam, n=6, p=2, seed=4)
    m, G, a, N = 2, 2, 0.7, 40000
    theta = prob.theta_bar + scale * np.array([1.5, -1.2])
    states = np.array(list(itertools.product(range(prob.n), repeat=m)), dtype=np.int64)
    est = O.loglik_batch(prob, m, G, np.tile(theta, (len(states), 1)), states, grad=False)
    log_pi = a * est["ell"] - 0.5 * a * a * est["sigma2"]
    pi = np.exp(log_pi - log_pi.max())
    pi /= pi.sum()
    rng = np.random.default_rng(1)
    us = states[rng.choice(len(states), size=N, p=pi)].copy()
    th = np.tile(theta, (N, 1))
    accepted = []
    for move in range(10):
        accepted.append(O.upm_move(prob, m, G, 31, 2, move, a, th, us).mean())
    assert 0.3 < np.mean(accepted) < 0.95  # proposals are really refused and taken
    counts = np.bincount(us[:, 0] * prob.n + us[:, 1], minlength=len(states))
    expect = N * pi
    big = expect >= 5
    obs, exp = counts[big], expect[big]
    if (~big).any():
        obs, exp = np.append(obs, counts[~big].sum()), np.append(exp, expect[~big].sum())
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-3
