"""GB300 (sm_103a) library for likelihood-annealed subsampling SMC (arXiv:1805.03317).

The compute path is the CUDA library built from ``csrc/`` and declared in ``include/subsmc.h``;
this package is its Python binding (``smc``) and build script (``build``).
"""
from .smc import (Batch, Context, SubsampledLoglik, SubsampledSMC, loglik_bwd, loglik_est, loglik_fwd,
                  loglik_full, loglik_grad, smc_autotune, smc_cv_moments,
                  smc_free, smc_get_cache, smc_get_centre, smc_get_mass, smc_get_particles,
                  smc_get_status, smc_init, smc_launch_count, smc_move, smc_move_adaptive,
                  smc_profile_enable,
                  smc_profile_read, smc_resample, smc_resample_noalloc,
                  smc_reweight, smc_set_particles, smc_set_scalars, smc_stage, smc_batch_init,
                  smc_batch_free, smc_batch_stage, smc_batch_autotune, smc_batch_tile, smc_batch_hmc_kernel,
                  smc_batch_launch_count, smc_batch_context, smc_batch_last_error,
                  smc_shard_export, smc_shard_import, smc_shard_gather_u, smc_shard_scatter_u,
                  smc_move_accepts, smc_finish_moves)
from .sharded import ShardedSMC, shard_bounds

__all__ = ["Batch", "smc_batch_init", "smc_batch_free", "smc_batch_stage", "smc_batch_autotune",
           "smc_batch_tile", "smc_batch_hmc_kernel", "smc_batch_launch_count", "smc_batch_context", "smc_batch_last_error",
           "Context", "SubsampledLoglik", "SubsampledSMC", "loglik_bwd", "loglik_est", "loglik_fwd",
           "loglik_full", "loglik_grad", "smc_autotune",
           "smc_cv_moments", "smc_free", "smc_get_cache", "smc_get_centre", "smc_get_mass",
           "smc_get_particles", "smc_get_status", "smc_init", "smc_launch_count", "smc_move",
           "smc_move_adaptive",
           "smc_profile_enable", "smc_profile_read", "smc_resample_noalloc",
           "smc_resample", "smc_reweight", "smc_set_particles", "smc_set_scalars", "smc_stage",
           "smc_shard_export", "smc_shard_import", "smc_shard_gather_u", "smc_shard_scatter_u",
           "smc_move_accepts", "smc_finish_moves", "ShardedSMC", "shard_bounds"]
