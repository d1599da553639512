"""Shared set-up for the GPU parity tests: the same seeded workload goes to the CUDA library (through
its C ABI) and to the FP64 oracle. The oracle computes its own control-variate centre; the GPU is
given that centre (rounded to the state precision for FP32/BF16 runs, and the oracle then uses the
rounded value too), so both sides expand around exactly the same theta_bar."""
import numpy as np
import torch

from oracle import oracle as O


def device_arrays(wl, dev="cuda:0"):
    if wl.x_dtype == "bf16":
        X = torch.from_numpy(wl.X_store.view(np.int16)).view(torch.bfloat16)
    else:
        X = torch.from_numpy(wl.X_store)
    return X.to(dev), torch.from_numpy(wl.y_store).to(dev)


def state_round(v, x_dtype):
    v = np.asarray(v, dtype=np.float64)
    return v if x_dtype == "f64" else v.astype(np.float32).astype(np.float64)


def oracle_problem(wl, theta_bar=None):
    prob = O.Problem(wl.family, wl.X, wl.y, wl.prior_mean, wl.prior_var, sigma=wl.sigma,
                     dof=wl.dof)
    tb = O.newton_map(prob) if theta_bar is None else np.asarray(theta_bar, np.float64)
    prob.set_centre(state_round(tb, wl.x_dtype))
    return prob


def make_pair(wl, theta_bar=None, tile_hint=0, **kw):
    import paper_1805_03317_gb300 as S
    prob = oracle_problem(wl, theta_bar)
    X, y = device_arrays(wl)
    args = dict(N=wl.N, m=wl.m, G=wl.G, L=wl.L, seed=wl.seed, noise_sigma=wl.sigma, dof=wl.dof,
                theta_bar=prob.theta_bar, tile_hint=tile_hint)
    args.update(kw)
    ctx = S.smc_init(X, y, wl.family, wl.prior_mean, wl.prior_var, **args)
    return prob, ctx


def tol(x_dtype):
    """Parity bars. FP64 runs: rounding-order only. FP32/BF16-stored runs compare with the oracle on
    the same stored values: log-likelihood estimate to 1e-5 relative, gradient to 1e-4 relative to
    its largest component; sigma2_hat to 1e-4 relative to its largest value plus the l_hat bar
    (it enters the log target in the same units as l_hat)."""
    if x_dtype == "f64":
        return dict(ell=1e-11, sig2=1e-8, grad=1e-9)
    return dict(ell=1e-5, sig2=1e-4, grad=1e-4)


def ell_scale(prob, theta, ell_ref):
    """Scale for the l_hat bar: the largest of |l_hat| and its four summands A, B'delta,
    delta'C delta/2 and (n/m) sum d (Sec. 3.2). Rounding acts on the summands, so a relative bar on
    an l_hat that nearly cancels is read against the largest summand."""
    import numpy as np
    d = np.asarray(theta, dtype=np.float64) - prob.theta_bar[None, :]
    A = np.full(d.shape[0], prob.A)
    Bd = d @ prob.B
    qC = 0.5 * np.einsum("bi,ij,bj->b", d, prob.C, d)
    rest = np.asarray(ell_ref) - A - Bd - qC
    return np.max(np.abs(np.stack([np.asarray(ell_ref), A, Bd, qC, rest])), axis=0)
