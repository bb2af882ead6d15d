"""ctypes mirror of include/dlx.h and the loader of the CUDA library.

The loader fails loudly: if the library is missing and cannot be built, or
no CUDA device is visible when a call needs one, an exception is raised.
There is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

DLX_OK, DLX_PENDING = 0, 1
DLX_ERR = {-1: "INVALID_ARG", -2: "NOMEM", -3: "CUDA", -4: "NONFINITE", -5: "TIMEOUT", -6: "RANGE",
           -7: "UNSUPPORTED"}
DLX_FP32_SIMT, DLX_TF32X3, DLX_BF16X3, DLX_BF16, DLX_BF16X4, DLX_F16X3, DLX_BF16X3SA = 0, 1, 2, 3, 4, 5, 6
PRECISIONS = {"fp32": DLX_FP32_SIMT, "tf32x3": DLX_TF32X3, "bf16x3": DLX_BF16X3, "bf16": DLX_BF16, "bf16x4": DLX_BF16X4,
              "f16x3": DLX_F16X3, "bf16x3sa": DLX_BF16X3SA}

_fp = C.POINTER(C.c_float)


class MftDesc(C.Structure):
    _fields_ = [("n_pupil", C.c_int), ("diameter_m", C.c_double), ("n_det", C.c_int), ("pixscale_rad", C.c_double),
                ("oversample", C.c_int), ("n_lambda", C.c_int), ("lambda_m", C.POINTER(C.c_double)),
                ("n_src", C.c_int), ("n_exp", C.c_int), ("n_zern", C.c_int), ("precision", C.c_int),
                ("psf_chunk", C.c_int), ("workspace_limit_bytes", C.c_size_t), ("prf_prior_sigma", C.c_double),
                ("dither_px", C.POINTER(C.c_int32)), ("focal_length_m", C.c_double), ("focal_shift_m", C.c_double)]


class Params(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("transmission", "opd_fixed", "zern_basis", "zern_coeff", "opd_pix",
                                          "weights", "flux", "pos", "dither", "flat")]


class Grads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("d_zern", "d_opd_pix", "d_flat", "d_flux", "d_pos")]


class PlanInfo(C.Structure):
    _fields_ = [(k, C.c_int) for k in ("n_pupil", "n_det", "oversample", "n_out", "n_lambda", "n_src", "n_exp",
                                       "n_zern", "n_psf", "precision", "psf_chunk")] + [
        ("workspace_bytes", C.c_size_t), ("flop_forward", C.c_double), ("flop_loss_grad", C.c_double),
        ("gemm_tiles_stage2", C.c_int), ("n_mft_out", C.c_int)]


class KernelTimes(C.Structure):
    _fields_ = [("n_classes", C.c_int), ("name", C.c_char_p * 16), ("ms", C.c_double * 16),
                ("events", C.c_int64 * 16), ("launches", C.c_int64 * 16), ("total_launches", C.c_int64)]


class Request(C.Structure):
    _fields_ = [("desc", MftDesc)] + [(k, C.c_void_p) for k in (
        "transmission", "opd_fixed", "zern_basis", "weights", "dither", "zern_coeff", "opd_pix", "flux", "pos",
        "flat", "data")] + [("n_steps", C.c_int), ("lr", C.c_float * 5), ("adam_m", C.c_void_p),
                            ("adam_v", C.c_void_p), ("adam_step", C.c_int)]


class Result(C.Structure):
    _fields_ = [("loss", C.c_double)] + [(k, C.c_void_p) for k in (
        "zern_coeff", "opd_pix", "flux", "pos", "flat", "g_zern", "g_opd_pix", "g_flux", "g_pos", "g_flat")] + [
        ("queued_s", C.c_double), ("latency_s", C.c_double), ("steps_done", C.c_int), ("adam_m", C.c_void_p),
        ("adam_v", C.c_void_p), ("adam_step", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("rejected", C.c_uint64), ("active", C.c_int), ("queued", C.c_int), ("hbm_in_use", C.c_size_t),
                ("hbm_budget", C.c_size_t), ("evals", C.c_uint64), ("graph_launches", C.c_uint64),
                ("grouped_launches", C.c_uint64), ("midflight_admits", C.c_uint64), ("slot_moves", C.c_uint64)]


# Every symbol include/dlx.h declares, with (restype, argtypes).
SIGNATURES = {
    "dlx_make_mft": (C.c_int, [C.POINTER(MftDesc), C.c_int, C.POINTER(C.c_void_p)]),
    "dlx_destroy_plan": (C.c_int, [C.c_void_p]),
    "dlx_plan_get_info": (C.c_int, [C.c_void_p, C.POINTER(PlanInfo)]),
    "dlx_forward": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_void_p]),
    "dlx_model_jvp": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_uint32, C.c_double, C.c_void_p,
                                C.c_void_p, C.c_void_p]),
    "dlx_model_vjp": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_void_p, C.POINTER(Grads), C.c_void_p]),
    "dlx_model_vjp_jvp": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_uint32, C.c_double,
                                    C.POINTER(Grads), C.POINTER(Grads), C.c_void_p]),
    "dlx_nll_cotangent": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "dlx_fisher_gram": (C.c_int, [C.c_void_p, C.c_int, C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "dlx_psf": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_void_p]),
    "dlx_forward_noalloc": (C.c_int, [C.POINTER(MftDesc), C.POINTER(Params), C.c_void_p, C.c_void_p]),
    "dlx_loss_grad": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_void_p, C.POINTER(Grads),
                                C.c_void_p, C.c_void_p]),
    "dlx_plan_diagnostics": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "dlx_plan_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "dlx_set_checks": (C.c_int, [C.c_int]),
    "dlx_get_checks": (C.c_int, []),
    "dlx_check_buffer": (C.c_int, [C.c_void_p, C.c_size_t, C.c_int]),
    "dlx_check_loss_grad_args": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_void_p,
                                           C.POINTER(Grads), C.c_void_p]),
    "dlx_plan_inject_fault": (C.c_int, [C.c_void_p, C.c_int]),
    "dlx_plan_get_timing": (C.c_int, [C.c_void_p, C.POINTER(KernelTimes)]),
    "dlx_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_float, C.c_float,
                           C.c_float, C.c_float, C.c_int, C.c_void_p]),
    "dlx_server_create": (C.c_int, [C.c_int, C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]),
    "dlx_server_destroy": (C.c_int, [C.c_void_p]),
    "dlx_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "dlx_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double, C.POINTER(Result)]),
    "dlx_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "dlx_server_inject_fault": (C.c_int, [C.c_void_p, C.c_int]),
    "dlx_last_error": (C.c_char_p, []),
    "dlx_version": (C.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.lib_path()


def load(build_if_missing: bool = True):
    """Load libdlx (building it in-tree with nvcc when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.lib_path()
            if build_if_missing and not _build.up_to_date():
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"dlx CUDA library not found at {path}; run build() first")
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype, fn.argtypes = res, args
            _lib = lib
    return _lib


class DlxError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = load().dlx_last_error().decode(errors="replace")
        super().__init__(f"{where} failed: {DLX_ERR.get(code, code)}: {msg}")


def check(code: int, where: str) -> int:
    if code < 0:
        raise DlxError(code, where)
    return code
