"""ctypes declarations of the libca C ABI (include/ca.h).  Marshalling only."""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

CA_OK, CA_ERR_INVALID_ARG, CA_ERR_CUDA, CA_ERR_OOM = 0, 1, 2, 3
CA_ERR_TIMEOUT, CA_ERR_UNSUPPORTED, CA_ERR_ADMISSION, CA_ERR_STATE = 4, 5, 6, 7
CA_HYP_RANDOM, CA_HYP_EXHAUSTIVE = 0, 1
CA_NORM_2N, CA_NORM_NK, CA_NORM_RAW = 0, 1, 2
CA_SCORER_HAND, CA_SCORER_LEARNED, CA_SCORER_LEARNED_FALLBACK = 0, 1, 2
CA_SCORER_2D, CA_SCORER_2D_FALLBACK = 3, 4
CA_DUMP_CANDIDATES, CA_DUMP_HYPOTHESES, CA_DUMP_TABLES = 1, 2, 3
CA_BATCH_AUTO, CA_BATCH_STAGED, CA_BATCH_FUSED = 0, 1, 2
CA_DUMP_LEARNED = 4
CA_DUMP_TRACE = 5
CA_SCORER_NPARAM = 17601
CA_SCORER2D_NPARAM = 6209
CA_LR_CONSTANT, CA_LR_COSINE = 0, 1
LUT_G, LUT_T, LUT_I = 5772, 8193, 256


class CaParams(C.Structure):
    _fields_ = [
        ("n_strips", C.c_int32), ("cands_per_strip", C.c_int32), ("n_hyps", C.c_int32),
        ("refine_iters", C.c_int32), ("alpha", C.c_float), ("t_g", C.c_float),
        ("t_theta_deg", C.c_float), ("t_iota", C.c_float), ("t_ps", C.c_float),
        ("t_cs", C.c_float), ("t_px", C.c_float), ("t_ri", C.c_float), ("r_min", C.c_float),
        ("r_max", C.c_float), ("d_max", C.c_float), ("sup_px", C.c_int32),
        ("hyp_mode", C.c_int32), ("score_norm", C.c_int32), ("sobel_norm", C.c_int32),
        ("scorer_mode", C.c_int32), ("hyp_threads", C.c_int32), ("batch_mode", C.c_int32),
        ("wave_frames", C.c_int32), ("prior_centre", C.c_int32), ("reserved", C.c_int32),
        ("seed", C.c_uint64),
    ]


class CaFrame(C.Structure):
    _fields_ = [("rgb_dev", C.c_void_p), ("mask_dev", C.c_void_p), ("H", C.c_int32),
                ("W", C.c_int32), ("pitch", C.c_int64), ("frame_key", C.c_uint64)]


class CaTuning(C.Structure):
    _fields_ = [("batch_mode", C.c_int32), ("hyp_threads", C.c_int32),
                ("wave_frames", C.c_int32), ("n_tried", C.c_int32), ("ms", C.c_float),
                ("ms_staged", C.c_float), ("ms_fused", C.c_float), ("ms_untuned", C.c_float),
                ("fit_lag", C.c_int32), ("mask_lag", C.c_int32)]


class CaTrainParams(C.Structure):
    _fields_ = [("lr", C.c_float), ("momentum", C.c_float), ("pos_weight", C.c_float),
                ("apply", C.c_int32), ("clip_norm", C.c_float), ("lr_schedule", C.c_int32)]


class CaSmoothParams(C.Structure):
    _fields_ = [("gamma", C.c_float), ("jump", C.c_float), ("t_hold", C.c_float),
                ("reserved", C.c_int32)]


class CaResult(C.Structure):
    _fields_ = [("cx", C.c_float), ("cy", C.c_float), ("r", C.c_float), ("score", C.c_float),
                ("valid", C.c_int32), ("n_inliers", C.c_int32)]


class CaServerConfig(C.Structure):
    _fields_ = [("params", CaParams), ("mem_budget", C.c_size_t), ("max_streams", C.c_int32),
                ("max_batch", C.c_int32), ("track", C.c_int32), ("want_masks", C.c_int32),
                ("smooth", C.c_int32), ("smooth_params", CaSmoothParams),
                ("zero_copy", C.c_int32), ("reserved", C.c_int32)]


class CaServerRequest(C.Structure):
    _fields_ = [("frame_host", C.c_void_p), ("mask_host", C.c_void_p), ("frame_key", C.c_uint64),
                ("t_arrival", C.c_double), ("stream_id", C.c_int32), ("H", C.c_int32),
                ("W", C.c_int32), ("reserved", C.c_int32)]


class CaServerResult(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("stream_id", C.c_int32), ("status", C.c_int32),
                ("frame_key", C.c_uint64), ("result", CaResult), ("t_arrival", C.c_double),
                ("t_submit", C.c_double), ("t_launch", C.c_double), ("t_done", C.c_double)]


# (name, restype, argtypes) of every exported function, in header order.
_P = C.POINTER
SIGNATURES = [
    ("ca_params_default", None, [_P(CaParams)]),
    ("ca_create", C.c_int, [_P(C.c_void_p), C.c_int]),
    ("ca_destroy", C.c_int, [C.c_void_p]),
    ("ca_estimate", C.c_int, [C.c_void_p, _P(CaFrame), C.c_int, _P(CaParams), C.c_void_p,
                              C.c_void_p]),
    ("ca_estimate_uniform", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                      _P(C.c_uint64), _P(CaParams), C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    ("ca_estimate_tracked", C.c_int, [C.c_void_p, _P(CaFrame), C.c_int, _P(CaParams), C.c_void_p,
                                      _P(C.c_int32), C.c_int, C.c_void_p, C.c_void_p]),
    ("ca_estimate_static", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, _P(C.c_uint64),
                                     _P(CaParams), C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ca_tune", C.c_int, [C.c_void_p, _P(CaFrame), C.c_int, _P(CaParams), C.c_void_p,
                          C.c_void_p, _P(CaTuning)]),
    ("ca_plan_create", C.c_int, [C.c_void_p, _P(CaFrame), C.c_int, _P(CaParams), C.c_void_p,
                                 _P(C.c_void_p)]),
    ("ca_plan_launch", C.c_int, [C.c_void_p, C.c_void_p]),
    ("ca_plan_destroy", C.c_int, [C.c_void_p]),
    ("ca_scorer_init", C.c_int, [C.c_void_p, C.c_uint64]),
    ("ca_scorer_set_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("ca_scorer_get_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("ca_scorer_save", C.c_int, [C.c_void_p, C.c_char_p]),
    ("ca_scorer_load", C.c_int, [C.c_void_p, C.c_char_p]),
    ("ca_scorer_forward", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ca_scorer_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_int, C.c_int, C.c_int, _P(CaTrainParams), _P(C.c_float),
                                 C.c_void_p]),
    ("ca_scorer_train", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                  C.c_int, _P(CaTrainParams), C.c_int, C.c_int, C.c_uint64,
                                  C.c_void_p]),
    ("ca_server_now", C.c_double, []),
    ("ca_server_create", C.c_int, [C.c_void_p, _P(CaServerConfig), _P(C.c_void_p)]),
    ("ca_server_submit", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_uint64,
                                   C.c_double, C.c_void_p, _P(C.c_uint64)]),
    ("ca_server_submit_batch", C.c_int, [C.c_void_p, _P(CaServerRequest), C.c_int,
                                         _P(C.c_uint64), _P(C.c_int)]),
    ("ca_server_poll", C.c_int, [C.c_void_p, C.c_int, _P(CaServerResult), C.c_int,
                                 _P(C.c_int)]),
    ("ca_server_stats", C.c_int, [C.c_void_p, _P(C.c_size_t), _P(C.c_int32), _P(C.c_int32)]),
    ("ca_server_destroy", C.c_int, [C.c_void_p]),
    ("ca_pool_create", C.c_int, [C.c_size_t, C.c_size_t, _P(C.c_void_p)]),
    ("ca_pool_alloc", C.c_int, [C.c_void_p, C.c_size_t, _P(C.c_size_t)]),
    ("ca_pool_free", C.c_int, [C.c_void_p, C.c_size_t]),
    ("ca_pool_stats", C.c_int, [C.c_void_p, _P(C.c_size_t), _P(C.c_size_t)]),
    ("ca_pool_destroy", C.c_int, [C.c_void_p]),
    ("ca_scorer2d_init", C.c_int, [C.c_void_p, C.c_uint64]),
    ("ca_scorer2d_set_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("ca_scorer2d_get_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("ca_scorer2d_save", C.c_int, [C.c_void_p, C.c_char_p]),
    ("ca_scorer2d_load", C.c_int, [C.c_void_p, C.c_char_p]),
    ("ca_scorer2d_forward", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                      C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ca_scorer2d_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_int, C.c_int, C.c_int, _P(CaTrainParams), _P(C.c_float),
                                   C.c_void_p]),
    ("ca_scorer2d_train", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_int, C.c_int, _P(CaTrainParams), C.c_int, C.c_int,
                                    C.c_uint64, C.c_void_p]),
    ("ca_smooth_tracked", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, _P(C.c_int32),
                                    _P(C.c_int32), C.c_int, _P(CaSmoothParams), C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    ("ca_mask", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, _P(C.c_int32), _P(C.c_int32),
                          _P(C.c_void_p), C.c_void_p]),
    ("ca_run_host", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                              _P(C.c_uint64), _P(CaParams), C.c_void_p, C.c_void_p]),
    ("ca_run_host_zero_copy", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                        _P(C.c_uint64), _P(CaParams), C.c_void_p, C.c_void_p]),
    ("ca_sync", C.c_int, [C.c_void_p, C.c_void_p]),
    ("ca_set_debug", C.c_int, [C.c_void_p, C.c_int]),
    ("ca_set_wait_limit", C.c_int, [C.c_void_p, C.c_uint64]),
    ("ca_inject_failure", C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    ("ca_debug_dump", C.c_int, [C.c_void_p, C.c_int, C.c_int, _P(CaParams), C.c_void_p,
                                C.c_size_t, _P(C.c_size_t)]),
    ("ca_launch_count", C.c_uint64, [C.c_void_p]),
    ("ca_set_trace", C.c_int, [C.c_void_p, C.c_int]),
    ("ca_set_timing", C.c_int, [C.c_void_p, C.c_int]),
    ("ca_kernel_times", C.c_int, [C.c_void_p, _P(C.c_double), _P(C.c_int32)]),
    ("ca_status_string", C.c_char_p, [C.c_int]),
    ("ca_last_error", C.c_char_p, [C.c_void_p]),
]

_lib = None


class CaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libca status %d (%s): %s" % (status, STATUS_NAMES.get(status, "?"), msg))
        self.status = status


STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of memory",
                4: "timeout", 5: "unsupported", 6: "admission refused", 7: "invalid state"}


def lib() -> C.CDLL:
    """The loaded libca.  Raises if the library has not been built: there is
    no fallback implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libca.so is missing (%s); build it with "
                               "paper_2210_14771_gb300.build.build()" % LIB)
        L = C.CDLL(LIB)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, handle=None):
    if status != CA_OK:
        msg = lib().ca_last_error(handle).decode() if handle else ""
        raise CaError(status, msg)
