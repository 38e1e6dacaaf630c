"""ctypes mirror of include/leja.h and the loader of the in-tree libleja.so.

Loading fails loudly (ImportError) when the native library has not been built: there is no
Python fallback for any compute step.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libleja.so")

# ll_status
LL_OK = 0
STATUS_NAMES = {
    0: "LL_OK", 1: "LL_ERR_INVALID_ARG", 2: "LL_ERR_BAD_CSR", 3: "LL_ERR_BAD_BOUNDS",
    4: "LL_ERR_DD_NOT_CONVERGED", 5: "LL_ERR_QR_BREAKDOWN", 6: "LL_ERR_NONFINITE", 7: "LL_ERR_TIMEOUT",
    8: "LL_ERR_OOM", 9: "LL_ERR_CUDA", 10: "LL_ERR_UNSUPPORTED", 11: "LL_ERR_NO_FORWARD",
}
LL_F64, LL_F32 = 0, 1
LL_PREC_F64, LL_PREC_DF64, LL_PREC_F32_MIXED = 0, 1, 2
LL_PROBE_RADEMACHER, LL_PROBE_GAUSSIAN = 0, 1
LL_SVAL_CENTER, LL_SVAL_HALF_LMAX = 0, 1
LL_DD_AUTO, LL_DD_TABLE_Q = 0, 1
LL_GRAM_AUTO, LL_GRAM_TENSOR, LL_GRAM_DFLOAT = 0, 1, 2
LL_FUSE_AUTO, LL_FUSE_ON, LL_FUSE_OFF = 0, 1, 2
LL_REORDER_AUTO, LL_REORDER_NONE, LL_REORDER_DEGREE = 0, 1, 2
LL_STREAM_S, LL_STREAM_G, LL_STREAM_POWER = 0, 1, 2
LL_KERNEL_AUTO, LL_KERNEL_GATHER, LL_KERNEL_TMA, LL_KERNEL_BAND = 0, 1, 2, 3
LL_EST_HUTCHPP, LL_EST_HUTCHINSON = 0, 1
LL_INJECT_NONE, LL_INJECT_STALL = 0, 1
LL_NOALLOC_MAX_ROWS = 1 << 18


class ll_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colind", ctypes.c_void_p), ("values", ctypes.c_void_p), ("dtype", ctypes.c_int)]


class ll_bounds(ctypes.Structure):
    _fields_ = [("lmin", ctypes.c_double), ("lmax", ctypes.c_double)]


class ll_options(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int), ("probes", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("probe_kind", ctypes.c_int), ("precision", ctypes.c_int), ("sval_mode", ctypes.c_int),
                ("keep_for_backward", ctypes.c_int), ("rows_per_thread", ctypes.c_int),
                ("threads_per_block", ctypes.c_int), ("ckpt_stride", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("timeout_cycles", ctypes.c_int64), ("step_kernel", ctypes.c_int), ("estimator", ctypes.c_int),
                ("tol", ctypes.c_double), ("dd_scheme", ctypes.c_int), ("qr_gram", ctypes.c_int),
                ("reorder", ctypes.c_int)]


class ll_info(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("c", ctypes.c_double), ("gamma", ctypes.c_double),
                ("trace_q", ctypes.c_double), ("trace_res", ctypes.c_double), ("estimate", ctypes.c_double),
                ("taylor_terms", ctypes.c_int), ("k", ctypes.c_int), ("kernel_launches", ctypes.c_int),
                ("ms_probes", ctypes.c_float), ("ms_pass1", ctypes.c_float), ("ms_qr", ctypes.c_float),
                ("ms_pass2", ctypes.c_float), ("ms_total", ctypes.c_float), ("kernel_pass1", ctypes.c_int),
                ("kernel_pass2", ctypes.c_int), ("threads_pass1", ctypes.c_int), ("threads_pass2", ctypes.c_int),
                ("deg_max_pass1", ctypes.c_int), ("deg_max_pass2", ctypes.c_int), ("deg_mean_pass2", ctypes.c_double),
                ("kept_w_steps", ctypes.c_int), ("kept_w_steps_pass1", ctypes.c_int),
                ("kept_w_stride", ctypes.c_int), ("forward_id", ctypes.c_int64),
                ("pairs_pass1", ctypes.c_int), ("pairs_pass2", ctypes.c_int),
                ("rows_pass1", ctypes.c_int), ("rows_pass2", ctypes.c_int), ("batch_tuned", ctypes.c_int),
                ("reordered", ctypes.c_int), ("adjoint_fused", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_U64 = ctypes.c_uint64
_PD = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); every entry point declared in include/leja.h
SIGNATURES = {
    "ll_create": (_I, [ctypes.POINTER(_P)]),
    "ll_destroy": (None, [_P]),
    "ll_status_string": (ctypes.c_char_p, [_I]),
    "ll_last_error": (ctypes.c_char_p, [_P]),
    "ll_default_options": (None, [ctypes.POINTER(ll_options)]),
    "ll_set_step_config": (_I, [_P, _I, _I, _I]),
    "ll_set_keep_budget": (_I, [_P, _I64]),
    "ll_set_adjoint_fusion": (_I, [_P, _I]),
    "ll_trim_workspace": (_I, [_P]),
    "ll_debug_inject": (_I, [_P, _I]),
    "ll_leja_points": (_I, [_I, _PD]),
    "ll_divided_differences": (_I, [ll_bounds, _I, _I, _PD, ctypes.POINTER(_I)]),
    "ll_divided_differences_q": (_I, [ll_bounds, _I, _PD]),
    "ll_gershgorin": (_I, [_P, ctypes.POINTER(ll_csr), ctypes.POINTER(ll_bounds), _P]),
    "ll_power_lmax": (_I, [_P, ctypes.POINTER(ll_csr), _I, _U64, _PD, _P]),
    "ll_power_lmax_noalloc": (_I, [ctypes.POINTER(ll_csr), _I, _U64, _PD, _P]),
    "ll_probes": (_I, [_P, _I, _U64, _I, _I64, _I, _P, _I64, _P]),
    "ll_apply_poly": (_I, [_P, ctypes.POINTER(ll_csr), ll_bounds, _I, _I, _P, _I64, _I, _P, _I64, _P]),
    "ll_apply_poly_tol": (_I, [_P, ctypes.POINTER(ll_csr), ll_bounds, _I, _D, _I, _P, _I64, _I, _P, _I64,
                               ctypes.POINTER(_I), _P]),
    "ll_logdet_forward": (_I, [_P, ctypes.POINTER(ll_csr), ll_bounds, ctypes.POINTER(ll_options), _PD, _P]),
    "ll_logdet_forward_host": (_I, [_P, ctypes.POINTER(ll_csr), ll_bounds, ctypes.POINTER(ll_options), _PD, _P]),
    "ll_logdet_backward": (_I, [_P, ctypes.POINTER(ll_csr), _D, _P, _P]),
    "ll_logdet_backward_qr": (_I, [_P, ctypes.POINTER(ll_csr), _D, _P, _P]),
    "ll_param_grad": (_I, [_P, _P, _P, _I64, _I64, _I, _PD, _P]),
    "ll_logdet_batched": (_I, [_P, ctypes.POINTER(ll_csr), ctypes.POINTER(ll_bounds), _I,
                               ctypes.POINTER(ll_options), ctypes.POINTER(_I), _PD, _P]),
    "ll_logdet_sweep": (_I, [_P, ctypes.POINTER(ll_csr), _P, _I, _PD, ctypes.POINTER(ll_bounds),
                             ctypes.POINTER(_I), ctypes.POINTER(ll_options), _PD, _P]),
    "ll_gram": (_I, [_P, _I, _P, _I64, _I, _P, _I64, _I, _I64, _I, _P, _P]),
    "ll_get_info": (_I, [_P, ctypes.POINTER(ll_info)]),
    "ll_stop_degrees": (_I, [_P, _I, ctypes.POINTER(_I), _I, ctypes.POINTER(_I)]),
    "ll_kept_basis": (_I, [_P, _P, _I64, ctypes.POINTER(_I64), ctypes.POINTER(_I), ctypes.POINTER(_I), _P]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libleja.so (built in-tree by paper_2603_02207_gb300.build); raise if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libleja.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
