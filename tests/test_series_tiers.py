"""The logistic increment's cumulant series (csrc/device.cuh, row_incr): the kernels evaluate
d = -sum_{k=3}^{K} kappa_k D^k / k! and r = -sum kappa_k D^(k-1) / (k-1)! through kappa_10 for
|D| <= 1/2 in FP32 (1/20 in FP64), and through kappa_6 where the streamed kernels' warp has every
|D| <= 1/20. For each (K, largest |D|) the truncation stays within at most 1.1e-8 of w |D|^3 in d
and 1.2e-7 of w D^2 in r, against d and r from their definitions in 50-digit arithmetic over a
grid of s = sigma(eta_bar) and D. The kappa_k are the Bernoulli cumulants (derivatives of
K(t) = log(1 - s + s e^t) at 0), computed symbolically here; the kernels write them as
polynomials in w = s(1 - s) and q = 1 - 2s."""
import math

import pytest

sp = pytest.importorskip("sympy")
mpmath = pytest.importorskip("mpmath")

TIERS = [(6, 0.05), (10, 0.5)]


@pytest.fixture(scope="module")
def cumulants():
    t, s = sp.symbols("t s")
    K = sp.log(1 - s + s * sp.exp(t))
    out, d = {}, K
    for k in range(1, 11):
        d = sp.diff(d, t)
        if k >= 3:
            out[k] = sp.lambdify(s, sp.simplify(d.subs(t, 0)), "mpmath")
    return out


def test_cumulants_match_the_kernels_polynomials(cumulants):
    """kappa_3..kappa_10 as the kernels write them (w = s(1-s), q = 1-2s)."""
    poly = {
        3: lambda w, q: w * q,
        4: lambda w, q: w * (1 - 6 * w),
        5: lambda w, q: w * q * (1 - 12 * w),
        6: lambda w, q: w * (1 + w * (-30 + 120 * w)),
        7: lambda w, q: w * q * (1 + w * (-60 + 360 * w)),
        8: lambda w, q: w * (1 + w * (-126 + w * (1680 - 5040 * w))),
        9: lambda w, q: w * q * (1 + w * (-252 + w * (5040 - 20160 * w))),
        10: lambda w, q: w * (1 + w * (-510 + w * (17640 + w * (-151200 + 362880 * w)))),
    }
    mpmath.mp.dps = 50
    for sv in [0.01, 0.2, 0.5, 0.73, 0.999]:
        s = mpmath.mpf(sv)
        w, q = s * (1 - s), 1 - 2 * s
        for k in range(3, 11):
            assert abs(cumulants[k](s) - poly[k](w, q)) <= mpmath.mpf(10) ** -40 * (1 + abs(poly[k](w, q)))


@pytest.mark.parametrize("kmax,dmax", TIERS)
def test_series_tier_error_within_the_kappa10_bound(cumulants, kmax, dmax):
    mpmath.mp.dps = 50
    worst_d = worst_r = 0.0
    for sv in [1e-4, 0.02, 0.1, 0.3, 0.5, 0.7, 0.9, 0.98, 1 - 1e-4]:
        s = mpmath.mpf(sv)
        w = s * (1 - s)
        kap = {k: cumulants[k](s) for k in range(3, kmax + 1)}
        for frac in [-1.0, -0.63, -0.25, 0.1, 0.5, 0.81, 1.0]:
            D = mpmath.mpf(frac * dmax)
            Kt = mpmath.log(1 - s + s * mpmath.exp(D))
            d_ref = -(Kt - s * D - w * D * D / 2)
            r_ref = -(s * mpmath.exp(D) / (1 - s + s * mpmath.exp(D)) - s - w * D)
            d_ser = -sum(kap[k] * D ** k / math.factorial(k) for k in kap)
            r_ser = -sum(kap[k] * D ** (k - 1) / math.factorial(k - 1) for k in kap)
            worst_d = max(worst_d, float(abs(d_ser - d_ref) / (w * abs(D) ** 3)))
            worst_r = max(worst_r, float(abs(r_ser - r_ref) / (w * D * D)))
    assert worst_d <= 1.1e-8 and worst_r <= 1.2e-7, (worst_d, worst_r)
