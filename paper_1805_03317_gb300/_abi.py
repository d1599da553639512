"""ctypes declarations of the C ABI in include/subsmc.h (argument marshalling only).

Loading fails loudly when the compiled library is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_i32, c_i64, c_u64, c_d, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_double, ctypes.c_void_p)
c_dp = ctypes.POINTER(ctypes.c_double)
c_ip = ctypes.POINTER(ctypes.c_int32)

SMC_OK, SMC_ERR_ARG, SMC_ERR_CUDA, SMC_ERR_NONFINITE, SMC_ERR_TIMEOUT, SMC_ERR_OOM = 0, -1, -2, -3, -4, -5
FAMILY = {"logistic": 0, "probit": 1, "poisson": 2, "gaussian": 3, "student_t": 4}
DTYPE = {"f64": 0, "f32": 1, "bf16": 2}


class SmcProblem(ctypes.Structure):
    _fields_ = [("family", c_i32), ("n", c_i64), ("p", c_i32), ("X", c_vp), ("x_dtype", c_i32),
                ("x_ld", c_i64), ("y", c_vp), ("prior_mean", c_dp), ("prior_var", c_dp),
                ("noise_sigma", c_d), ("dof", c_d)]


class SmcConfig(ctypes.Structure):
    _fields_ = [("N", c_i32), ("m", c_i32), ("G", c_i32), ("L", c_i32), ("ess_frac", c_d),
                ("seed", c_u64), ("search_k", c_i32), ("search_rounds", c_i32), ("eps0", c_d),
                ("tile_hint", c_i32), ("hmc_kernel", c_i32), ("cv_kernel", c_i32),
                ("cv_order", c_i32), ("cv_centre", c_i32), ("full_data", c_i32),
                ("resampling", c_i32), ("grid_points", c_i32), ("grid_decades", c_d),
                ("theta_move", c_i32), ("eps_jitter", c_d), ("shard_base", c_i32),
                ("shard_count", c_i32)]


# name -> (restype, argtypes)
SIGNATURES = {
    "smc_init": (ctypes.c_int, [ctypes.POINTER(c_vp), ctypes.POINTER(SmcProblem),
                                ctypes.POINTER(SmcConfig), c_dp, c_vp]),
    "smc_free": (ctypes.c_int, [c_vp]),
    "smc_last_error": (ctypes.c_char_p, [c_vp]),
    "smc_reweight": (ctypes.c_int, [c_vp, c_dp, c_dp, c_dp]),
    "smc_resample": (ctypes.c_int, [c_vp, c_vp]),
    "smc_move": (ctypes.c_int, [c_vp, c_i32, c_dp, c_dp]),
    "smc_move_adaptive": (ctypes.c_int, [c_vp, c_i32, c_d, c_d, c_ip, c_dp, c_dp]),
    "smc_stage": (ctypes.c_int, [c_vp, c_i32, c_i32]),
    "smc_batch_init": (ctypes.c_int, [ctypes.POINTER(c_vp), c_i32, ctypes.POINTER(SmcProblem),
                                      ctypes.POINTER(SmcConfig), c_vp]),
    "smc_batch_free": (ctypes.c_int, [c_vp]),
    "smc_batch_last_error": (ctypes.c_char_p, [c_vp]),
    "smc_batch_context": (ctypes.c_int, [c_vp, c_i32, ctypes.POINTER(c_vp)]),
    "smc_batch_tile": (ctypes.c_int, [c_vp, ctypes.POINTER(c_i32)]),
    "smc_batch_hmc_kernel": (ctypes.c_int, [c_vp, c_i32, ctypes.POINTER(c_i32)]),
    "smc_batch_launch_count": (ctypes.c_int64, [c_vp]),
    "smc_batch_stage": (ctypes.c_int, [c_vp, c_i32, c_i32]),
    "smc_batch_autotune": (ctypes.c_int, [c_vp, ctypes.POINTER(c_i32)]),
    "loglik_est": (ctypes.c_int, [c_vp, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "loglik_grad": (ctypes.c_int, [c_vp, c_i32, c_vp, c_vp, c_d, c_vp, c_vp, c_vp]),
    "loglik_full": (ctypes.c_int, [c_vp, c_i32, c_vp, c_d, c_vp, c_vp]),
    "loglik_fwd": (ctypes.c_int, [c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "loglik_bwd": (ctypes.c_int, [c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "smc_get_particles": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp]),
    "smc_set_particles": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp]),
    "smc_get_cache": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp]),
    "smc_get_centre": (ctypes.c_int, [c_vp, c_dp, c_dp, c_dp, c_dp]),
    "smc_cv_moments": (ctypes.c_int, [c_vp, c_dp, c_dp, c_dp, c_dp]),
    "smc_get_mass": (ctypes.c_int, [c_vp, c_dp, c_dp]),
    "smc_get_status": (ctypes.c_int, [c_vp, c_dp, c_dp, c_ip, c_dp]),
    "smc_set_scalars": (ctypes.c_int, [c_vp, c_i32, c_d, c_d, c_d]),
    "smc_autotune": (ctypes.c_int, [c_vp, c_ip, c_ip]),
    "smc_launch_count": (ctypes.c_int64, [c_vp]),
    "smc_profile_enable": (ctypes.c_int, [c_vp, c_i32]),
    "smc_profile_read": (ctypes.c_int, [c_vp, c_i32, ctypes.POINTER(c_i64), c_dp]),
    "smc_resample_noalloc": (ctypes.c_int, [c_i32, c_vp, c_u64, c_i32, c_vp, c_vp]),
    "smc_shard_export": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "smc_shard_import": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "smc_shard_gather_u": (ctypes.c_int, [c_vp, c_i32, c_vp, c_vp, c_i32]),
    "smc_shard_scatter_u": (ctypes.c_int, [c_vp, c_i32, c_vp, c_vp]),
    "smc_move_accepts": (ctypes.c_int, [c_vp, ctypes.POINTER(c_u64), ctypes.POINTER(c_u64)]),
    "smc_finish_moves": (ctypes.c_int, [c_vp, c_i32, c_u64, c_u64]),
}
NOALLOC_MAX_N = 262144

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libsubsmc.so (optionally building it first). Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c \"import __graft_entry__ as g;"
                          f" g.build()\"` (sm_103a CUDA library; there is no CPU implementation)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SmcError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


def check(code: int, where: str, ctx=None) -> None:
    if code != SMC_OK:
        msg = load().smc_last_error(ctx)
        raise SmcError(code, where, (msg or b"").decode(errors="replace"))
