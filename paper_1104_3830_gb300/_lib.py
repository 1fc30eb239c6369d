"""ctypes binding of libsa (include/sa.h).  Argument marshalling only: every step of the
path runs inside the library.  Device buffers are torch CUDA tensors (data_ptr); the
library never sees torch types.

The library is built in-tree by ``paper_1104_3830_gb300.build`` (``__graft_entry__.build``)
and there is no fallback: if ``libsa.so`` is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsa.so")

SA_OK, SA_PENDING = 0, 1
SA_E_INVALID, SA_E_NOMEM, SA_E_CUDA, SA_E_NOT_CONVERGED = -1, -2, -3, -4
SA_E_NO_PERFECT_MATCHING, SA_E_NONFINITE, SA_E_BUDGET, SA_E_TIMEOUT, SA_E_UNSUPPORTED = -5, -6, -7, -8, -9
SA_I16, SA_I32 = 0, 1
OPTION = {"wait_limit_ns": 0, "solve_gpu": 1, "step_sparse": 2, "max_grid": 3, "fused_threads": 4, "step_l2_bytes": 5,
          "test_unreachable_barrier": 6}
SA_BATCH_BLOCK, SA_BATCH_GROUP, SA_BATCH_REGS, SA_BATCH_KROWS = 0, 1, 2, 3
PREC = {"mixed": 0, "fp32": 1, "fp64": 2}
KERNEL = {"auto": 0, "fused": 1, "plain": 2, "step": 3, "newton": 4}
STATUS_NAMES = {0: "SA_OK", 1: "SA_PENDING", -1: "SA_E_INVALID", -2: "SA_E_NOMEM", -3: "SA_E_CUDA",
                -4: "SA_E_NOT_CONVERGED", -5: "SA_E_NO_PERFECT_MATCHING", -6: "SA_E_NONFINITE",
                -7: "SA_E_BUDGET", -8: "SA_E_TIMEOUT", -9: "SA_E_UNSUPPORTED"}


class SaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sa_matrix(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p), ("wtype", ctypes.c_int), ("n", ctypes.c_int32), ("ld", ctypes.c_int64)]


class sa_scale_opts(ctypes.Structure):
    _fields_ = [("p", ctypes.POINTER(ctypes.c_double)), ("n_p", ctypes.c_int32), ("tol", ctypes.c_double),
                ("max_sweeps_per_p", ctypes.c_int32), ("prec", ctypes.c_int), ("kernel", ctypes.c_int),
                ("warm_keep_v", ctypes.c_int32), ("resume_from", ctypes.c_int32)]


class sa_scale_info(ctypes.Structure):
    _fields_ = [("sweeps_total", ctypes.c_int64), ("residual", ctypes.c_double), ("p_final", ctypes.c_double),
                ("converged", ctypes.c_int32), ("steps_done", ctypes.c_int32), ("fallback_rows", ctypes.c_int32),
                ("kernel_used", ctypes.c_int32), ("kernel_ms", ctypes.c_double),
                ("sparse_epochs", ctypes.c_int32), ("reanchors", ctypes.c_int32)]


class sa_batch_plan(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("n_hi", ctypes.c_int32 * 8), ("path", ctypes.c_int32 * 8),
                ("warps", ctypes.c_int32 * 8), ("per_block", ctypes.c_int32 * 8)]


class sa_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("col", ctypes.POINTER(ctypes.c_int32)), ("w", ctypes.POINTER(ctypes.c_int32))]


class sa_auction_info(ctypes.Structure):
    _fields_ = [("phases", ctypes.c_int32), ("rounds", ctypes.c_int64), ("complete", ctypes.c_int32),
                ("auction_sum_log_w", ctypes.c_double), ("eps_final", ctypes.c_double),
                ("auction_ms", ctypes.c_double), ("host_ms", ctypes.c_double),
                ("searches", ctypes.c_int64), ("search_rounds", ctypes.c_int64)]


class sa_assign_result(ctypes.Structure):
    _fields_ = [("perm", ctypes.POINTER(ctypes.c_int32)), ("sum_log_w", ctypes.c_double),
                ("log_ub", ctypes.c_double), ("gamma", ctypes.c_double), ("nnz_first", ctypes.c_int64),
                ("nnz_final", ctypes.c_int64), ("repairs", ctypes.c_int32), ("reprunes", ctypes.c_int32),
                ("scale", sa_scale_info), ("ms_scale", ctypes.c_double), ("ms_prune", ctypes.c_double),
                ("ms_solve", ctypes.c_double), ("ms_certify", ctypes.c_double)]


class sa_alg1_opts(ctypes.Structure):
    _fields_ = [("opt_ratio", ctypes.c_double), ("p0", ctypes.c_double), ("dp", ctypes.c_double),
                ("max_rounds", ctypes.c_int32), ("eps", ctypes.c_double), ("t", ctypes.c_double),
                ("max_sweeps_per_p", ctypes.c_int32), ("prec", ctypes.c_int), ("kernel", ctypes.c_int)]


class sa_alg1_result(ctypes.Structure):
    _fields_ = [("perm", ctypes.POINTER(ctypes.c_int32)), ("sum_log_w", ctypes.c_double), ("gamma", ctypes.c_double),
                ("p_final", ctypes.c_double), ("p_raw", ctypes.c_double), ("rounds", ctypes.c_int32),
                ("sweeps_total", ctypes.c_int64), ("nnz", ctypes.c_int64)]


class sa_result(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("perm", ctypes.POINTER(ctypes.c_int32)), ("sum_log_w", ctypes.c_double),
                ("gamma", ctypes.c_double), ("sweeps", ctypes.c_int64), ("status", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("t_scaled", ctypes.c_double)]


class sa_server_stats(ctypes.Structure):
    _fields_ = [("live_launches", ctypes.c_int64), ("live_requests", ctypes.c_int64),
                ("live_device_bytes", ctypes.c_int64), ("live_blocks", ctypes.c_int32),
                ("live_slots", ctypes.c_int32), ("live_capacity", ctypes.c_int32), ("large_grid", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()
_VP, _DP, _I32P, _I64P = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), \
    ctypes.POINTER(ctypes.c_int64)

SIGNATURES = {
    "sa_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]),
    "sa_destroy": (None, [_VP]),
    "sa_set_option": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int64]),
    "sa_set_batch_plan": (ctypes.c_int, [_VP, ctypes.c_void_p]),
    "sa_last_error": (ctypes.c_char_p, []),
    "sa_version": (ctypes.c_char_p, []),
    "sa_kernel_launches": (ctypes.c_int64, []),
    "sa_scale": (ctypes.c_int, [_VP, ctypes.POINTER(sa_matrix), ctypes.POINTER(sa_scale_opts), _VP, _VP,
                                ctypes.POINTER(sa_scale_info)]),
    "sa_scale_noalloc": (ctypes.c_int, [ctypes.POINTER(sa_matrix), ctypes.POINTER(sa_scale_opts), _VP, _VP, _VP,
                                        ctypes.POINTER(sa_scale_info)]),
    "sa_verify": (ctypes.c_int, [_VP, ctypes.POINTER(sa_matrix), ctypes.c_double, _VP, _VP, _VP, _VP, _DP, _DP]),
    "sa_prune": (ctypes.c_int, [_VP, ctypes.POINTER(sa_matrix), ctypes.c_double, _VP, _VP, ctypes.c_double,
                                ctypes.c_int32, ctypes.POINTER(sa_csr), _DP]),
    "sa_solve_reduced": (ctypes.c_int, [ctypes.POINTER(sa_csr), _I32P, _DP, _DP, _DP]),
    "sa_solve_reduced_warm": (ctypes.c_int, [ctypes.POINTER(sa_csr), _DP, _I32P, _DP, _DP, _DP]),
    "sa_solve_reduced_near": (ctypes.c_int, [ctypes.POINTER(sa_csr), _DP, _I32P, _DP, _DP, _DP]),
    "sa_solve_reduced_gpu": (ctypes.c_int, [_VP, ctypes.POINTER(sa_csr), _DP, _I32P, _DP, _DP, _DP,
                                            ctypes.POINTER(sa_auction_info)]),
    "sa_certify": (ctypes.c_int, [_VP, ctypes.POINTER(sa_matrix), _DP, _DP, ctypes.c_double, _I64P,
                                  ctypes.c_int64, ctypes.POINTER(sa_csr)]),
    "sa_csr_free": (None, [ctypes.POINTER(sa_csr)]),
    "sa_assign": (ctypes.c_int, [_VP, ctypes.POINTER(sa_matrix), ctypes.POINTER(sa_scale_opts), ctypes.c_double,
                                 ctypes.POINTER(sa_assign_result)]),
    "sa_assign_host": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int32, ctypes.c_int64,
                                      ctypes.POINTER(sa_scale_opts), ctypes.c_double,
                                      ctypes.POINTER(sa_assign_result)]),
    "sa_algorithm1": (ctypes.c_int, [_VP, ctypes.POINTER(sa_matrix), ctypes.POINTER(sa_alg1_opts),
                                     ctypes.POINTER(sa_alg1_result)]),
    "sa_narrow_i32_to_i16": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, ctypes.c_int64, ctypes.c_int32, _I64P]),
    "sa_batch_scale": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, ctypes.c_int,
                                      ctypes.POINTER(sa_scale_opts), _VP, _VP, _I32P, _I32P]),
    "sa_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t,
                                        ctypes.POINTER(sa_scale_opts), ctypes.c_int32]),
    "sa_server_destroy": (None, [_VP]),
    "sa_submit": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]),
    "sa_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(sa_result)]),
    "sa_result_release": (None, [_VP, ctypes.c_uint64]),
    "sa_server_now": (ctypes.c_double, [_VP]),
    "sa_server_request_bytes": (ctypes.c_size_t, [_VP, ctypes.c_int, ctypes.c_int32]),
    "sa_debug_fail_allocs": (None, [ctypes.c_int32]),
    "sa_server_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(sa_server_stats)]),
}


def lib():
    """The loaded libsa (raises if it was not built: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libsa.so is not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype, f.argtypes = res, args
            _lib = L
        return _lib


def check(status):
    if status not in (SA_OK, SA_PENDING):
        msg = lib().sa_last_error().decode(errors="replace")
        raise SaError(status, msg)
    return status


def make_opts(p, tol=1e-6, max_sweeps=20000, prec="mixed", kernel="auto", warm_keep_v=False, resume_from=0):
    parr = np.ascontiguousarray(np.atleast_1d(p), dtype=np.float64)
    o = sa_scale_opts(parr.ctypes.data_as(_DP), len(parr), float(tol), int(max_sweeps), PREC[prec], KERNEL[kernel],
                      int(bool(warm_keep_v)), int(resume_from))
    o._keep = parr  # keep the schedule alive with the struct
    return o


def info_dict(info: sa_scale_info) -> dict:
    return {k: getattr(info, k) for k, _ in sa_scale_info._fields_}
