"""smc_resample_noalloc: systematic resampling for callers that cannot allocate device memory
(for example code running inside CUDA graph capture, or a host with a fixed memory arena).

It must return exactly the ancestors that smc_resample returns on a context set for systematic
resampling (the default; the entry point has no multinomial variant) for the same weights, seed
and stage, on consecutive calls (its scratch array is shared and reused from call to call), and it
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


def test_noalloc_matches_context_resampling_at_the_largest_size():
    """N = SMC_NOALLOC_MAX_N with skewed (non-uniform) weights: every entry of the scratch array is
    used, and the ancestors equal those of smc_resample on a context of that many particles."""
    import paper_1805_03317_gb300 as S
    from gpu_common import make_pair
    from paper_1805_03317_gb300._abi import NOALLOC_MAX_N
    from smc_workloads import small_glm

    N = NOALLOC_MAX_N
    wl = small_glm("logistic", n=2000, p=2, N=N, m=2, G=1, L=1, x_dtype="f32", seed=6)
    prob, ctx = make_pair(wl)
    dev = "cuda:0"
    rng = np.random.default_rng(2)
    W = rng.random(N) ** 8
    W[rng.integers(0, N, size=50)] *= 1e3  # a few heavy particles with many offspring
    W /= W.sum()
    th = (prob.theta_bar + 0.1 * rng.standard_normal((N, wl.p))).astype(np.float32)
    u = rng.integers(0, wl.n, size=(N, wl.m))
    S.smc_set_particles(ctx, torch.from_numpy(th).to(dev), torch.from_numpy(u).to(dev),
                        torch.from_numpy(W).to(dev))
    for stage in (3, 17):
        S.smc_set_scalars(ctx, stage, 0.5, 0.3, 0.0)
        S.smc_set_particles(ctx, None, None, torch.from_numpy(W).to(dev))
        anc_ctx = torch.empty(N, dtype=torch.int32, device=dev)
        S.smc_resample(ctx, anc_ctx)
        anc = torch.full((N,), -1, dtype=torch.int32, device=dev)
        S.smc_resample_noalloc(torch.from_numpy(W).to(dev), wl.seed, stage, anc)
        torch.cuda.synchronize()
        assert torch.equal(anc, anc_ctx), f"stage {stage}"
        counts = torch.bincount(anc.long(), minlength=N).cpu().numpy()
        assert counts.max() > 1 and (counts == 0).any()  # the weights really were uneven
    S.smc_free(ctx)
