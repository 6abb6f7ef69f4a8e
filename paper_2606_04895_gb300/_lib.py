"""ctypes binding of libbst.so (include/bst.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_STATE, ERR_CUDA, ERR_NOT_PD, ERR_TIMEOUT, ERR_NONFINITE, ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_STATE", "ERR_CUDA", "ERR_NOT_PD", "ERR_TIMEOUT", "ERR_NONFINITE",
                "ERR_UNSUPPORTED"]
MH, MALA, HMC, NUTS, AIES, AIES_DE, NUTS_MULTINOMIAL = range(7)
BF16, FP32, FP64, FP16 = range(4)
LIK_EMULATOR, LIK_ANALYTIC = range(2)

# Every symbol include/bst.h declares.
SYMBOLS = [
    "bst_version", "bst_last_error", "bst_create", "bst_destroy", "bst_set_emulator", "bst_get_emulator", "bst_set_emulator_output",
    "bst_set_analytic", "bst_init_chains", "bst_step", "bst_loglike", "bst_grad_loglike", "bst_welford_reset",
    "bst_welford_add", "bst_adapt_cov", "bst_get_state", "bst_set_state", "bst_get_whitening", "bst_get_counters",
    "bst_train_step", "bst_train_grad", "bst_ess", "bst_draw_positions", "bst_set_whitening", "bst_set_bounds_penalty", "bst_r_minus_1", "bst_r_minus_1_parts", "bst_r_minus_1_combine", "bst_quantiles", "bst_credible_metric", "bst_sliced_wasserstein", "bst_sync", "bst_grad_loglike_noalloc",
    "bst_welford_stats", "bst_welford_merge", "bst_train_apply",
]


class BstError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


class Config(C.Structure):
    _fields_ = [
        ("d", C.c_int), ("n_chains", C.c_int), ("precision", C.c_int), ("lik_kind", C.c_int),
        ("seed", C.c_uint64), ("max_depth", C.c_int), ("aies_walkers", C.c_int), ("aies_a", C.c_double),
        ("thin", C.c_int), ("device", C.c_int),
    ]


class StepStats(C.Structure):
    _fields_ = [
        ("accepts", C.c_int64), ("evals", C.c_int64), ("divergences", C.c_int64), ("accept_stat", C.c_double),
        ("status", C.c_int),
    ]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libbst.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libbst.so not found at {_build.LIB}; run paper_2606_04895_gb300.build.build()")
        L = C.CDLL(_build.LIB)
        vp, i, d, u32p = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_uint32)
        h = vp
        L.bst_version.restype = C.c_char_p
        L.bst_last_error.restype = C.c_char_p
        L.bst_create.argtypes = [C.POINTER(vp), C.POINTER(Config)]
        L.bst_destroy.argtypes = [h]
        L.bst_destroy.restype = None
        L.bst_set_emulator.argtypes = [h, i, i, vp, vp, vp, d, d]
        L.bst_get_emulator.argtypes = [h, vp]
        L.bst_set_emulator_output.argtypes = [h, i, d]
        L.bst_set_analytic.argtypes = [h, i, i, i, vp, vp, vp, vp, vp, d, i]
        L.bst_init_chains.argtypes = [h, vp, vp, vp, vp, vp, vp]
        L.bst_step.argtypes = [h, i, d, i, i, vp, vp, C.POINTER(StepStats)]
        L.bst_loglike.argtypes = [h, vp, i, vp, vp]
        L.bst_grad_loglike.argtypes = [h, vp, i, vp, vp, vp]
        L.bst_welford_reset.argtypes = [h]
        L.bst_welford_add.argtypes = [h, vp, i, vp]
        L.bst_adapt_cov.argtypes = [h, d, vp, vp, vp]
        L.bst_get_state.argtypes = [h, vp, vp, vp, vp]
        L.bst_set_state.argtypes = [h, vp, vp, vp, vp]
        L.bst_get_whitening.argtypes = [h, vp, vp]
        L.bst_get_counters.argtypes = [h, vp, vp, vp, vp]
        L.bst_train_step.argtypes = [h, vp, vp, i, d, d, d, d, vp, vp]
        L.bst_train_grad.argtypes = [h, vp, vp, i, vp, vp, vp]
        L.bst_ess.argtypes = [h, vp, i, vp]
        L.bst_r_minus_1.argtypes = [h, vp, i, vp]
        L.bst_set_whitening.argtypes = [h, vp, vp]
        L.bst_set_bounds_penalty.argtypes = [h, vp]
        L.bst_draw_positions.argtypes = [h, i, vp, vp, vp, vp, vp]
        L.bst_quantiles.argtypes = [h, vp, i, vp, i, vp]
        L.bst_credible_metric.argtypes = [h, vp, i, C.c_double, vp, vp, vp]
        L.bst_r_minus_1_parts.argtypes = [h, vp, i, vp, vp]
        L.bst_r_minus_1_combine.argtypes = [i, i, i, vp, vp, vp]
        L.bst_sliced_wasserstein.argtypes = [h, vp, i, vp, C.c_longlong, i, C.c_ulonglong, vp]
        L.bst_sync.argtypes = [h, vp]
        L.bst_grad_loglike_noalloc.argtypes = [h, vp, i, vp, vp, vp]
        L.bst_welford_stats.argtypes = [h, vp, vp, vp]
        L.bst_welford_merge.argtypes = [h, d, vp, vp]
        L.bst_train_apply.argtypes = [h, vp, d, d, d, d, vp]
        for name in SYMBOLS:
            if name not in ("bst_version", "bst_last_error", "bst_destroy"):
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def check(status: int):
    if status != OK:
        msg = load(False).bst_last_error().decode(errors="replace")
        raise BstError(status, msg)
