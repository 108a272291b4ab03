"""ctypes declarations of the libhawkes C ABI (include/hawkes.h).

Loading fails loudly when the in-tree library is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhawkes.so")

HAWKES_OK = 0
STATUS_NAMES = {
    0: "HAWKES_OK",
    1: "HAWKES_ERR_INVALID_ARG",
    2: "HAWKES_ERR_ZERO_RATE",
    3: "HAWKES_ERR_CUDA",
    5: "HAWKES_ERR_OOM",
    6: "HAWKES_ERR_INVALID_DATA",
}
PREC = {"mixed": 0, "fp64": 1}
OPTIONS = {"block_warps": 1, "ctas_per_sm": 2, "profile": 3, "times_sorted": 4, "mixed_fixup_exp": 5,
           "skip_far_blocks": 6, "fp64_ordered": 7, "col_groups": 8, "one_launch": 9,
           "partial_slots": 10, "bmds_fused": 11}

# every function declared in include/hawkes.h
EXPORTED = (
    "hawkes_ctx_create", "hawkes_ctx_destroy", "hawkes_last_error", "hawkes_ctx_sync_status",
    "hawkes_ctx_set_option", "hawkes_ctx_kernel_stats", "hawkes_ctx_reset_stats", "hawkes_loglik",
    "hawkes_loglik_grad_locations", "hmc_leapfrog_trajectory", "hawkes_batch_loglik_grad", "hawkes_version",
    "hawkes_ctx_launch_count", "hawkes_probe_pipe_rates", "hawkes_loglik_noalloc", "hawkes_ctx_set_tuning",
    "hawkes_ctx_get_tuning", "hawkes_autotune", "hawkes_batch_hmc_trajectory", "hawkes_self_excitation_prob",
    "hawkes_bmds_loglik_grad", "hawkes_bmds_workspace_bytes", "hawkes_mwg_create", "hawkes_mwg_destroy",
    "hawkes_mwg_last_error", "hawkes_mwg_delta", "hawkes_mwg_step", "hawkes_mwg_refresh", "hawkes_mwg_read",
    "hawkes_mwg_sync_status", "hawkes_mwg_propose_circle", "hawkes_mwg_propose_box", "hawkes_bmds_hmc_trajectory",
    "hawkes_mwg_set_precision", "hawkes_probe_dfma_rate", "hawkes_probe_exp2_fp64",
)
NOALLOC_MAX_N = 8192  # HAWKES_NOALLOC_MAX_N


class HawkesParams(ctypes.Structure):
    """Theta = (mu0, tau_x, tau_t, theta, omega, h) in the paper's order."""

    _fields_ = [(n, ctypes.c_double) for n in ("mu0", "tau_x", "tau_t", "theta", "omega", "h")]


class HawkesError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None


def _declare(lib: ctypes.CDLL) -> ctypes.CDLL:
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    pp = ctypes.POINTER(HawkesParams)
    st = ctypes.c_int
    lib.hawkes_ctx_create.argtypes = [ctypes.POINTER(vp), i32, i64, i32]
    lib.hawkes_ctx_create.restype = st
    lib.hawkes_ctx_destroy.argtypes = [vp]
    lib.hawkes_ctx_destroy.restype = None
    lib.hawkes_last_error.argtypes = [vp]
    lib.hawkes_last_error.restype = ctypes.c_char_p
    lib.hawkes_ctx_sync_status.argtypes = [vp, vp]
    lib.hawkes_ctx_sync_status.restype = st
    lib.hawkes_ctx_set_option.argtypes = [vp, i32, i64]
    lib.hawkes_ctx_set_option.restype = st
    lib.hawkes_ctx_kernel_stats.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                            ctypes.POINTER(ctypes.c_double)]
    lib.hawkes_ctx_kernel_stats.restype = st
    lib.hawkes_ctx_launch_count.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.hawkes_ctx_launch_count.restype = st
    lib.hawkes_ctx_reset_stats.argtypes = [vp]
    lib.hawkes_ctx_reset_stats.restype = st
    lib.hawkes_self_excitation_prob.argtypes = [vp, dp, dp, i64, i32, pp, i32, vp, dp]
    lib.hawkes_self_excitation_prob.restype = st
    lib.hawkes_bmds_loglik_grad.argtypes = [vp, dp, i32, dp, i64, i32, ctypes.c_double, i32, vp, dp, dp, dp]
    lib.hawkes_bmds_loglik_grad.restype = st
    lib.hawkes_bmds_workspace_bytes.argtypes = [i64, i32, i32]
    lib.hawkes_bmds_workspace_bytes.restype = ctypes.c_size_t
    lib.hawkes_mwg_create.argtypes = [i32, dp, dp, i64, i32, pp, i32, vp, ctypes.POINTER(vp)]
    lib.hawkes_mwg_create.restype = st
    lib.hawkes_mwg_destroy.argtypes = [vp]
    lib.hawkes_mwg_destroy.restype = None
    lib.hawkes_mwg_last_error.argtypes = [vp]
    lib.hawkes_mwg_last_error.restype = ctypes.c_char_p
    lib.hawkes_mwg_delta.argtypes = [vp, i32, dp, dp, vp, dp]
    lib.hawkes_mwg_delta.restype = st
    lib.hawkes_mwg_step.argtypes = [vp, i32, dp, dp, dp, dp, vp, dp, dp]
    lib.hawkes_mwg_step.restype = st
    lib.hawkes_mwg_refresh.argtypes = [vp, vp]
    lib.hawkes_mwg_refresh.restype = st
    lib.hawkes_mwg_set_precision.argtypes = [vp, ctypes.c_int, vp]
    lib.hawkes_mwg_set_precision.restype = st
    lib.hawkes_mwg_read.argtypes = [vp, vp, dp, dp, dp]
    lib.hawkes_mwg_read.restype = st
    lib.hawkes_mwg_propose_circle.argtypes = [vp, i32, dp, dp, dp, ctypes.c_double, i32, dp, vp, dp, dp]
    lib.hawkes_mwg_propose_circle.restype = st
    lib.hawkes_mwg_propose_box.argtypes = [vp, i32, dp, dp, dp, ctypes.c_double, dp, vp, dp, dp]
    lib.hawkes_mwg_propose_box.restype = st
    lib.hawkes_mwg_sync_status.argtypes = [vp, vp]
    lib.hawkes_mwg_sync_status.restype = st
    lib.hawkes_loglik.argtypes = [vp, dp, dp, i64, i32, pp, i32, vp, dp]
    lib.hawkes_loglik.restype = st
    lib.hawkes_loglik_grad_locations.argtypes = [vp, dp, dp, i64, i32, pp, i32, vp, dp, dp, dp]
    lib.hawkes_loglik_grad_locations.restype = st
    lib.hmc_leapfrog_trajectory.argtypes = [vp, dp, dp, dp, dp, dp, i64, i32, pp, ctypes.c_double, i32, dp, i32,
                                            vp, dp, dp, dp]
    lib.hmc_leapfrog_trajectory.restype = st
    lib.hawkes_bmds_hmc_trajectory.argtypes = [vp, dp, dp, dp, i64, i32, pp, dp, i32, ctypes.c_double,
                                               ctypes.c_double, i32, dp, i32, vp, dp, dp, dp]
    lib.hawkes_bmds_hmc_trajectory.restype = st
    lib.hawkes_batch_loglik_grad.argtypes = [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i32), dp, dp, pp, i32,
                                             vp, dp, dp]
    lib.hawkes_batch_loglik_grad.restype = st
    lib.hawkes_batch_hmc_trajectory.argtypes = [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i32), dp, dp, dp, dp,
                                                dp, pp, ctypes.POINTER(ctypes.c_double), i32, dp, i32, vp, dp, dp,
                                                dp]
    lib.hawkes_batch_hmc_trajectory.restype = st
    ip = ctypes.POINTER(i32)
    lib.hawkes_ctx_set_tuning.argtypes = [vp, i32, i32, i32, i32, i32]
    lib.hawkes_ctx_set_tuning.restype = st
    lib.hawkes_ctx_get_tuning.argtypes = [vp, i32, i32, ip, ip, ip]
    lib.hawkes_ctx_get_tuning.restype = st
    lib.hawkes_autotune.argtypes = [vp, dp, dp, i64, i32, pp, vp, ip, ip, ip, ctypes.POINTER(ctypes.c_double)]
    lib.hawkes_autotune.restype = st
    lib.hawkes_loglik_noalloc.argtypes = [dp, dp, i64, i32, pp, vp, dp]
    lib.hawkes_loglik_noalloc.restype = st
    dpp = ctypes.POINTER(ctypes.c_double)
    lib.hawkes_probe_pipe_rates.argtypes = [i32, dpp, dpp, dpp]
    lib.hawkes_probe_pipe_rates.restype = st
    lib.hawkes_probe_dfma_rate.argtypes = [i32, dpp]
    lib.hawkes_probe_dfma_rate.restype = st
    lib.hawkes_probe_exp2_fp64.argtypes = [vp, vp, i64, vp]
    lib.hawkes_probe_exp2_fp64.restype = st
    lib.hawkes_version.argtypes = []
    lib.hawkes_version.restype = ctypes.c_char_p
    return lib


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libhawkes.so (built by ``build.py``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libhawkes.so not found at {p}; build it with paper_2010_02994_gb300/build.py")
            _lib = _declare(ctypes.CDLL(p))
        return _lib
