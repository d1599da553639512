"""The synthetic input recipe (host logic, no GPU): each generator produces the shapes, value
distributions and storage the workloads are specified with, deterministically from its seed."""
import math

import numpy as np
import pytest
from scipy import interpolate

import smc_workloads as W


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 1e-3, 3.0e38], dtype=np.float32)
    bits = W.round_to_bf16_bits(x)
    back = W.bf16_bits_to_f64(bits)
    # ties go to the even mantissa; values already representable are exact
    assert back[0] == 1.0 and back[3] == -2.5
    assert back[1] == 1.0                        # halfway between 1 and 1 + 2^-7: even (1)
    assert back[2] == 1.0 + 2 ** -7              # above halfway: rounds up
    assert np.all(np.abs(back - x) <= np.abs(x) * 2.0 ** -8)


def test_generators_are_deterministic():
    a = W.small_glm("poisson", n=500, p=4, seed=9, x_scale=0.3)
    b = W.small_glm("poisson", n=500, p=4, seed=9, x_scale=0.3)
    assert np.array_equal(a.X_store, b.X_store) and np.array_equal(a.y_store, b.y_store)


def test_logistic_headline_workload_shape():
    wl = W.logistic_1e6("bf16", n=200_000)
    assert wl.X_store.shape == (200_000, 20) and wl.x_dtype == "bf16"
    X = wl.X
    assert np.all(X[:, 0] == 1.0)
    # AR(1) correlation 0.5 between neighbouring covariates, unit variances
    assert abs(np.corrcoef(X[:, 5], X[:, 6])[0, 1] - 0.5) < 0.01
    assert abs(np.corrcoef(X[:, 5], X[:, 7])[0, 1] - 0.25) < 0.01
    assert np.all(np.abs(X[:, 1:].var(axis=0) - 1.0) < 0.02)
    assert set(np.unique(wl.y)) <= {0.0, 1.0}
    assert (wl.N, wl.m, wl.G, wl.L, wl.R) == (4096, 1000, 10, 20, 5)


def test_student_t_workload_matches_the_papers_design():
    """Sec. 4.3: 50 covariates with unit variances and pairwise correlation 0.9, theta ~ U(-5, 5),
    t_5 errors, prior N(0, 10 I), sample fraction 0.0025, G = 100."""
    wl = W.student_t_5e5("f32", n=100_000)
    X = wl.X
    assert X.shape == (100_000, 50)
    C = np.corrcoef(X.T)
    off = C[~np.eye(50, dtype=bool)]
    assert abs(off.mean() - 0.9) < 0.01 and np.all(np.abs(np.diag(np.cov(X.T)) - 1.0) < 0.03)
    assert np.all(np.abs(wl.theta_true) <= 5.0)
    e = wl.y - X @ wl.theta_true
    # t_5: variance 5/3 and excess kurtosis 6
    assert abs(e.var() - 5.0 / 3.0) < 0.05
    k = np.mean((e - e.mean()) ** 4) / e.var() ** 2 - 3.0
    assert 3.0 < k < 12.0
    assert wl.m == 1250 and wl.G == 100 and np.all(wl.prior_var == 10.0) and wl.dof == 5.0


def test_gam_basis_is_the_clamped_cubic_bspline_partition_of_unity():
    u = np.linspace(0.0, 1.0, 500, endpoint=False)
    B = W.gam_basis(u[:, None]).astype(np.float64)
    assert B.shape == (500, 10)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-6)
    # against scipy's B-spline basis on the same knots
    for j in range(10):
        c = np.zeros(10)
        c[j] = 1.0
        ref = interpolate.BSpline(W.GAM_KNOTS, c, 3, extrapolate=False)(u)
        np.testing.assert_allclose(B[:, j], np.nan_to_num(ref), atol=1e-6)


def test_batch_workloads_are_uneven_and_clamped():
    wls = W.batch_uneven(P=12, N=64, n_lo=10_000, n_hi=1_000_000, upcast=False)
    ns = np.array([w.n for w in wls])
    ps = np.array([w.X_store.shape[1] for w in wls])
    assert np.all((ns >= 10_000) & (ns <= 1_000_000)) and len(set(ns)) == 12
    assert np.all((ps >= 5) & (ps <= 40))
    for w in wls:
        assert w.family in ("logistic", "probit")
        assert w.m == min(1000, max(100, math.ceil(w.n / 1000)))
