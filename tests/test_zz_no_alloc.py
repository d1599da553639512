"""smc_resample_noalloc: systematic resampling for callers that cannot allocate device memory
(for example code running inside CUDA graph capture, or a host with a fixed memory arena).

It must return exactly the ancestors that smc_resample returns for the same weights, seed and
stage, on consecutive calls (its scratch array is shared and reused from call to call), and it
must refuse sizes beyond its fixed scratch with an argument error. Resampling is integer work,
so the comparison is bit-exact. This file is collected last on purpose."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_resampling_matches_context_resampling_on_consecutive_calls():
    import paper_1805_03317_gb300 as S
    from gpu_common import make_pair
    from smc_workloads import small_glm

    wl = small_glm("logistic", n=2000, p=3, N=3001, m=8, G=2, L=1, x_dtype="f64", seed=5)
    prob, ctx = make_pair(wl)
    rng = np.random.default_rng(1)
    dev = "cuda:0"
    for call, stage in enumerate((4, 11)):
        W = rng.random(wl.N) ** (3 + 2 * call)
        W /= W.sum()
        th = prob.theta_bar + 0.1 * rng.standard_normal((wl.N, wl.p))
        u = rng.integers(0, wl.n, size=(wl.N, wl.m))
        S.smc_set_particles(ctx, torch.from_numpy(th).to(dev), torch.from_numpy(u).to(dev),
                            torch.from_numpy(W).to(dev))
        S.smc_set_scalars(ctx, stage, 0.5, 0.3, 0.0)
        anc_ctx = torch.empty(wl.N, dtype=torch.int32, device=dev)
        S.smc_resample(ctx, anc_ctx)
        W_dev = torch.from_numpy(W).to(dev)
        anc = torch.full((wl.N,), -1, dtype=torch.int32, device=dev)
        S.smc_resample_noalloc(W_dev, wl.seed, stage, anc)
        torch.cuda.synchronize()
        assert torch.equal(anc, anc_ctx), f"call {call}"
        assert int(anc.min()) >= 0 and int(anc.max()) < wl.N
    S.smc_free(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1805_03317_gb300 as S
    from paper_1805_03317_gb300._abi import NOALLOC_MAX_N, SmcError

    n = NOALLOC_MAX_N + 1
    W = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda:0")
    anc = torch.empty(n, dtype=torch.int32, device="cuda:0")
    with pytest.raises(SmcError) as e:
        S.smc_resample_noalloc(W, 1, 1, anc)
    assert e.value.code == -1
    # the largest accepted size works and gives the identity for uniform weights
    n = NOALLOC_MAX_N
    W = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda:0")
    anc = torch.empty(n, dtype=torch.int32, device="cuda:0")
    S.smc_resample_noalloc(W, 1, 1, anc)
    torch.cuda.synchronize()
    assert torch.equal(anc, torch.arange(n, dtype=torch.int32, device="cuda:0"))
