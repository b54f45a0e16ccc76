"""ctypes declarations of the C ABI in include/love.h.

Loading fails loudly: there is no fallback implementation of any call.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblove.so")

LOVE_OK = 0
STATUS_NAMES = {0: "LOVE_OK", 1: "LOVE_ERR_ARG", 2: "LOVE_ERR_DOMAIN", 3: "LOVE_ERR_NOT_PD",
                4: "LOVE_ERR_NAN", 5: "LOVE_ERR_OOM", 6: "LOVE_ERR_CUDA", 7: "LOVE_ERR_TIMEOUT",
                8: "LOVE_ERR_STATE", 9: "LOVE_ERR_UNSUPPORTED"}
F32, F64, BF16 = 0, 1, 2
WANT_MEAN, WANT_SAMPLER, WANT_GRAD, PRIOR_EXACT, TIME_REORTH = 0x1, 0x2, 0x4, 0x8, 0x10
BATCH_STREAMS = 0x20

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class love_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class love_ski_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int64), ("grid_size", C.c_int64 * 3),
                ("grid_lo", C.c_double * 3), ("grid_hi", C.c_double * 3),
                ("outputscale", C.c_double), ("lengthscale", C.c_double * 3),
                ("noise", C.c_double), ("dtype", C.c_int),
                ("allocator", C.POINTER(love_allocator)), ("additive", C.c_int)]


class love_precompute_opts(C.Structure):
    _fields_ = [("k", C.c_int), ("cache_dtype", C.c_int), ("flags", C.c_uint),
                ("breakdown_tol", C.c_double), ("cg_tol", C.c_double),
                ("cg_max_iter", C.c_int), ("sampler_k", C.c_int),
                ("sampler_seed", C.c_uint64), ("reorth", C.c_int), ("reorth_eta", C.c_double),
                ("cg_plain", C.c_int)]


class love_cache_info_t(C.Structure):
    _fields_ = [("dim", C.c_int), ("grid_size", C.c_int64 * 3), ("m", C.c_int64),
                ("k_eff", C.c_int), ("ld", C.c_int), ("sampler_k", C.c_int),
                ("cg_iters", C.c_int), ("sampler_fallback", C.c_int), ("dtype", C.c_int),
                ("cache_dtype", C.c_int), ("flags", C.c_uint), ("phase_ms", C.c_float * 4),
                ("reorth_skipped", C.c_int), ("reorth_ms", C.c_float),
                ("batched_rows", C.c_int)]


class love_device_status_t(C.Structure):
    _fields_ = [("bits", C.c_uint32), ("domain_errors", C.c_int64), ("clamped", C.c_int64)]


class love_batch_info_t(C.Structure):
    _fields_ = [("lanes_per_point", C.c_int), ("ctas_per_sm", C.c_int), ("n_candidates", C.c_int),
                ("candidate_ms", C.c_float * 16), ("chunks", C.c_int64), ("graph_captures", C.c_int64),
                ("graph_captures_dropped", C.c_int64)]


VP = C.c_void_p
DP = C.POINTER(C.c_double)

# name -> (restype, argtypes); the list of every exported entry point
SIGNATURES = {
    "ski_build": (C.c_int, [C.POINTER(love_ski_desc), VP, VP, VP, C.POINTER(VP)]),
    "ski_destroy": (C.c_int, [VP]),
    "ski_mvm": (C.c_int, [VP, VP, VP, VP]),
    "ski_mvm_kuu": (C.c_int, [VP, VP, VP, VP]),
    "ski_mvm_kuu_noalloc": (C.c_int, [VP, VP, VP, VP]),
    "love_precompute": (C.c_int, [VP, C.POINTER(love_precompute_opts), VP, C.POINTER(VP),
                                  C.POINTER(C.c_int)]),
    "love_cache_destroy": (C.c_int, [VP]),
    "love_predict_mean_var": (C.c_int, [VP, C.c_int64, VP, VP, VP, VP]),
    "love_predict_mean_var_host": (C.c_int, [VP, C.c_int64, VP, VP, VP, VP]),
    "love_sample": (C.c_int, [VP, C.c_int64, VP, C.c_int, VP, C.c_uint64, VP, VP]),
    "love_predict_var_root": (C.c_int, [VP, C.c_int64, VP, VP, VP]),
    "love_predict_covariance": (C.c_int, [VP, C.c_int64, VP, C.c_int64, VP, VP, VP]),
    "love_sampler_precompute": (C.c_int, [VP, C.c_int, C.c_uint64, VP]),
    "love_var_backward": (C.c_int, [VP, C.c_int64, VP, VP, VP, DP, DP, VP]),
    "love_cache_info": (C.c_int, [VP, C.POINTER(love_cache_info_t)]),
    "love_cache_import": (C.c_int, [C.POINTER(love_ski_desc), C.c_int, C.c_int, C.c_uint, DP, DP,
                                    C.c_int, DP, DP, DP, DP, VP, C.POINTER(VP)]),
    "love_cache_export": (C.c_int, [VP, DP, DP, DP, DP, DP, DP, VP]),
    "love_cache_save": (C.c_int, [VP, C.c_char_p, VP]),
    "love_cache_load": (C.c_int, [C.c_char_p, C.POINTER(love_allocator), VP, C.POINTER(VP)]),
    "love_get_device_status": (C.c_int, [VP, C.c_int, C.POINTER(love_device_status_t), VP]),
    "love_precompute_batched": (C.c_int, [C.c_int, C.POINTER(VP), C.POINTER(love_precompute_opts), C.c_int, VP,
                                          C.POINTER(VP), C.POINTER(C.c_int)]),
    "love_batch_create": (C.c_int, [C.c_int, C.POINTER(VP), C.POINTER(C.c_int64), VP, C.POINTER(VP)]),
    "love_batch_destroy": (C.c_int, [VP]),
    "love_predict_batched": (C.c_int, [VP, VP, VP, VP, VP]),
    "love_sample_batched": (C.c_int, [VP, VP, C.c_int, C.c_uint64, VP, VP]),
    "love_batch_serve": (C.c_int, [VP, VP, VP, VP, C.c_int, C.c_uint64, VP, C.c_int, VP]),
    "love_batch_info": (C.c_int, [VP, C.POINTER(love_batch_info_t)]),
    "love_status_string": (C.c_char_p, [C.c_int]),
    "love_last_cuda_error": (C.c_int, []),
    "love_launch_count": (C.c_uint64, []),
    "love_version": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load liblove.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(nvcc, sm_103a).  There is no CPU fallback.")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LoveError(RuntimeError):
    def __init__(self, call: str, status: int):
        self.status = status
        lib = _lib
        msg = lib.love_status_string(status).decode() if lib else ""
        extra = ""
        if status == 6 and lib:
            extra = f" (cudaError {lib.love_last_cuda_error()})"
        super().__init__(f"{call} -> {STATUS_NAMES.get(status, status)}: {msg}{extra}")


def check(call: str, status: int):
    if status != LOVE_OK:
        raise LoveError(call, status)
