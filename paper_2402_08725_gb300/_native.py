"""ctypes declarations of the C ABI in include/starred.h (argument marshalling only).

The library must have been built (``paper_2402_08725_gb300.build.build()``);
there is no fallback: loading fails loudly when the shared object is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int, c_double, c_float, c_size_t, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.c_size_t, ctypes.c_void_p
c_int64 = ctypes.c_int64
P_float = ctypes.POINTER(c_float)
P_double = ctypes.POINTER(c_double)

SR_MAX_GROUPS = 8
STATUS = {0: "SR_OK", 1: "SR_ERR_ARG", 2: "SR_ERR_SHAPE", 3: "SR_ERR_STATE", 4: "SR_ERR_CUDA", 5: "SR_ERR_OOM",
          6: "SR_ERR_NONFINITE", 7: "SR_ERR_TIMEOUT", 8: "SR_ERR_UNSUPPORTED"}
SR_DECONV, SR_PSF = 0, 1
SR_CONV_AUTO, SR_CONV_DIRECT, SR_CONV_PLAIN, SR_CONV_FFT = 0, 1, 2, 3
SR_ADABELIEF, SR_ADAM = 0, 1


class ProblemDesc(ctypes.Structure):
    _fields_ = [("kind", c_int), ("n_epochs", c_int), ("data_n", c_int), ("supersampling", c_int),
                ("psf_k", c_int), ("n_sources", c_int), ("n_scales", c_int), ("lam", c_double),
                ("conv_mode", c_int)]


class Layout(ctypes.Structure):
    _fields_ = [("n_groups", c_int), ("offset", c_size_t * SR_MAX_GROUPS), ("count", c_size_t * SR_MAX_GROUPS),
                ("total", c_size_t)]


class NoiseTiming(ctypes.Structure):
    _fields_ = [("draw_ms", c_double), ("corr_ms", c_double), ("starlet_ms", c_double), ("final_ms", c_double),
                ("launches", c_int), ("batch", c_int)]


class LbfgsbCfg(ctypes.Structure):
    _fields_ = [("m", c_int), ("max_iter", c_int), ("max_ls", c_int), ("pgtol", c_double), ("factr", c_double)]


class LbfgsbInfo(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("evaluations", c_int), ("status", c_int), ("f", c_double),
                ("pg_norm", c_double)]


LBFGSB_STATUS = {0: "pgtol", 1: "factr", 2: "max_iter", 3: "line_search"}


class OptimCfg(ctypes.Structure):
    _fields_ = [("kind", c_int), ("beta1", c_float), ("beta2", c_float), ("eps", c_float),
                ("lr", c_float * SR_MAX_GROUPS)]


# name -> (argtypes, restype); the same set of names as the header's declarations
PROTOTYPES = {
    "sr_last_error": ([], ctypes.c_char_p),
    "sr_version": ([], c_int),
    "sr_build_arch": ([], c_int),
    "sr_create_problem": ([ctypes.POINTER(ProblemDesc), c_void_p, ctypes.POINTER(c_void_p)], c_int),
    "sr_destroy": ([c_void_p], c_int),
    "sr_set_data": ([c_void_p, c_void_p, c_int], c_int),
    "sr_set_noise": ([c_void_p, c_void_p, c_int], c_int),
    "sr_set_psfs": ([c_void_p, c_void_p, c_int], c_int),
    "sr_set_weights": ([c_void_p, c_void_p], c_int),
    "sr_param_count": ([c_void_p], c_size_t),
    "sr_param_layout": ([c_void_p, ctypes.POINTER(Layout)], c_int),
    "sr_loss": ([c_void_p, c_void_p, P_double], c_int),
    "sr_loss_and_grad": ([c_void_p, c_void_p, P_double, c_void_p, c_void_p], c_int),
    "sr_loss_and_grad_host": ([c_void_p, c_void_p, P_double, c_void_p], c_int),
    "sr_loss_and_grad_host_async": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "sr_sync": ([c_void_p], c_int),
    "sr_step": ([c_void_p, c_void_p, c_int, ctypes.POINTER(OptimCfg), c_void_p, P_double], c_int),
    "sr_reset_optimizer": ([c_void_p], c_int),
    "sr_get_state": ([c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_int64)], c_int),
    "sr_set_state": ([c_void_p, c_void_p, c_void_p, c_int64], c_int),
    "sr_batch_create": ([ctypes.POINTER(c_void_p), c_int, c_void_p, ctypes.POINTER(c_void_p)], c_int),
    "sr_batch_destroy": ([c_void_p], c_int),
    "sr_batch_param_count": ([c_void_p], c_size_t),
    "sr_batch_param_offset": ([c_void_p, c_int, ctypes.POINTER(c_size_t)], c_int),
    "sr_batch_loss_and_grad": ([c_void_p, c_void_p, c_void_p, c_void_p, P_double, c_void_p], c_int),
    "sr_batch_loss_and_grad_host": ([c_void_p, c_void_p, P_double, c_void_p], c_int),
    "sr_batch_loss_and_grad_host_async": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "sr_batch_sync": ([c_void_p], c_int),
    "sr_batch_step": ([c_void_p, c_void_p, c_int, ctypes.POINTER(OptimCfg), P_double], c_int),
    "sr_batch_reset_optimizer": ([c_void_p], c_int),
    "sr_launches_per_eval": ([c_void_p], c_int),
    "sr_batch_launches_per_eval": ([c_void_p], c_int),
    "sr_batch_field_form": ([c_void_p, c_int], c_int),
    "sr_batch_set_schedule": ([c_void_p, c_int, c_int], c_int),
    "sr_batch_get_schedule": ([c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int)], c_int),
    "sr_batch_tune_schedule": ([c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_float)],
                               c_int),
    "sr_batch_profile": ([c_void_p, c_int], c_int),
    "sr_batch_profile_read": ([c_void_p, ctypes.POINTER(c_int), P_double, P_double, P_double], c_int),
    "sr_measure_fp32_peak": ([P_double], c_int),
    "sr_set_lambda_pts": ([c_void_p, c_double], c_int),
    "sr_set_translate_h": ([c_void_p, c_int], c_int),
    "sr_set_rotations": ([c_void_p, P_double], c_int),
    "sr_set_weight_map": ([c_void_p, c_void_p, c_int], c_int),
    "sr_psf_model": ([c_void_p, c_void_p, c_void_p], c_int),
    "sr_batch_set_data": ([c_void_p, c_void_p, c_int], c_int),
    "sr_batch_set_noise": ([c_void_p, c_void_p, c_int], c_int),
    "sr_batch_set_psfs": ([c_void_p, c_void_p, c_int], c_int),
    "sr_batch_lbfgsb": ([c_void_p, c_void_p, ctypes.POINTER(LbfgsbCfg), P_double, ctypes.POINTER(LbfgsbInfo)], c_int),
    "sr_batch_lbfgsb_fields": ([c_void_p, c_void_p, ctypes.POINTER(LbfgsbCfg), P_double, ctypes.POINTER(LbfgsbInfo),
                                ctypes.POINTER(c_int)], c_int),
    "sr_lbfgsb": ([c_void_p, c_void_p, ctypes.POINTER(LbfgsbCfg), P_double, ctypes.POINTER(LbfgsbInfo)], c_int),
    "sr_estimate_lambda_pts": ([c_void_p, c_void_p, P_double], c_int),
    "sr_noise_weights": ([c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_int, ctypes.c_uint64, P_float,
                          c_void_p, ctypes.POINTER(NoiseTiming), c_void_p], c_int),
    "sr_loss_and_grad_noalloc": ([ctypes.POINTER(ProblemDesc), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p], c_int),
}

_lock = threading.Lock()
_lib = None


class StarredError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


def load(path: str | None = None, build_if_missing: bool = True):
    """Load (building first if needed) the shared library and declare its prototypes."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if path is None:
            path = _build.lib_path()
            if build_if_missing:
                path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run paper_2402_08725_gb300.build)")
        lib = ctypes.CDLL(path)
        for name, (args, res) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def check(code: int, what: str):
    if code != 0:
        msg = load().sr_last_error().decode(errors="replace")
        raise StarredError(code, what, msg)
