"""Reference posterior quantities of the plain logistic workload (n = 10,000, p = 5, prior N(0, 10 I))
by importance sampling, computed with numpy/scipy only (no oracle, no CUDA library): the Bernoulli
log-likelihood and normal prior written out directly, and a multivariate-t (5 degrees of freedom)
proposal centred at the posterior mode with the Laplace covariance. It gives the log marginal
likelihood log p(y) (Sec. 3.5's target of the SMC estimate) and the posterior mean and standard
deviations, against which whole SMC runs of that workload are checked."""
from __future__ import annotations

import math

import numpy as np
from scipy import special, stats


def logistic_log_post(X, y, prior_var, th):
    """log p(y | theta) + log p(theta) for a batch th [B, p] (the prior's normalising constant
    included)."""
    eta = X @ th.T
    ll = (y[:, None] * eta - np.logaddexp(0.0, eta)).sum(axis=0)
    lp = stats.norm.logpdf(th, 0.0, np.sqrt(prior_var)).sum(axis=1)
    return ll + lp


def logistic_mode_and_laplace(X, y, prior_var, iters=50):
    """Posterior mode by Newton's method and the inverse negative Hessian there (numpy only)."""
    p = X.shape[1]
    th = np.zeros(p)
    for _ in range(iters):
        s = special.expit(X @ th)
        g = X.T @ (y - s) - th / prior_var
        H = -(X.T * (s * (1.0 - s))) @ X - np.diag(1.0 / prior_var)
        step = np.linalg.solve(-H, g)
        th = th + step
        if np.max(np.abs(step)) < 1e-12:
            break
    s = special.expit(X @ th)
    H = -(X.T * (s * (1.0 - s))) @ X - np.diag(1.0 / prior_var)
    return th, np.linalg.inv(-H)


def importance_reference(X, y, prior_var, M=40000, seed=0, nu=5.0, chunk=2000):
    """log p(y), the posterior mean and posterior sd by importance sampling with a t_nu proposal at
    the mode with the Laplace covariance. Returns a dict with the estimates and the relative
    standard error of the estimate of p(y)."""
    mode, Sig = logistic_mode_and_laplace(X, y, prior_var)
    p = X.shape[1]
    rng = np.random.default_rng(seed)
    Lc = np.linalg.cholesky(Sig)
    q = stats.multivariate_t(loc=mode, shape=Sig, df=nu)
    logw, ths = [], []
    for _ in range(M // chunk):
        z = rng.standard_normal((chunk, p))
        g = rng.chisquare(nu, chunk)
        th = mode + (z @ Lc.T) / np.sqrt(g / nu)[:, None]
        logw.append(logistic_log_post(X, y, prior_var, th) - q.logpdf(th))
        ths.append(th)
    logw = np.concatenate(logw)
    ths = np.concatenate(ths)
    log_ml = float(special.logsumexp(logw) - math.log(M))
    w = np.exp(logw - special.logsumexp(logw))
    mean = w @ ths
    sd = np.sqrt(w @ (ths - mean) ** 2)
    rel_se = math.sqrt(np.var(np.exp(logw - log_ml)) / M)
    return {"log_ml": log_ml, "mean": mean, "sd": sd, "rel_se": rel_se, "mode": mode}
