"""ctypes declarations of the C ABI in include/rf.h (argument marshalling only).

The library is the in-tree librfgpu.so produced by build.py.  Loading fails
loudly when it is missing: there is no CPU fallback."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librfgpu.so")

RF_OK, RF_E_INVALID, RF_E_OOM, RF_E_CUDA, RF_E_DOMAIN, RF_E_NOT_CONVERGED, RF_E_TIMEOUT = range(7)
STATUS_NAMES = {0: "RF_OK", 1: "RF_E_INVALID", 2: "RF_E_OOM", 3: "RF_E_CUDA", 4: "RF_E_DOMAIN",
                5: "RF_E_NOT_CONVERGED", 6: "RF_E_TIMEOUT"}
KIND = {"obs": 0, "param": 1, "gauss": 2, "exp": 3, "gaussexp": 4, "cheb": 5, "poly": 6, "sum": 7, "prod": 8,
        "poisson": 9, "extend": 10, "expr": 11}
RF_F64, RF_F32 = 0, 1


class rf_modifier(C.Structure):
    _fields_ = [("sample", C.c_int32), ("kind", C.c_int32), ("param", C.c_int32), ("k_lo", C.c_double),
                ("k_hi", C.c_double)]


class rf_node(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_in", C.c_int32), ("in_", C.c_int32 * 8), ("value", C.c_double),
                ("lo", C.c_double), ("hi", C.c_double), ("is_free", C.c_int32)]


class rf_expr(C.Structure):
    _fields_ = [("node", C.c_int32), ("n_ops", C.c_int32), ("ops", C.POINTER(C.c_int32)), ("n_consts", C.c_int32),
                ("consts", C.POINTER(C.c_double))]


class rf_fit_opts(C.Structure):
    _fields_ = [("tol_edm", C.c_double), ("max_evals", C.c_int32), ("want_cov", C.c_int32),
                ("no_graph", C.c_int32), ("host_steps", C.c_int32)]


# Every exported symbol of include/rf.h with (restype, argtypes).
_vp, _dp, _ip, _i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
SIGNATURES = {
    "rf_model_create": (C.c_int, [C.POINTER(rf_node), C.c_int32, C.c_int32, C.POINTER(_vp)]),
    "rf_model_create_expr": (C.c_int, [C.POINTER(rf_node), C.c_int32, C.c_int32, C.POINTER(rf_expr), C.c_int32,
                                       C.POINTER(_vp)]),
    "rf_model_destroy": (None, [_vp]),
    "rf_model_n_free": (C.c_int32, [_vp]),
    "rf_model_n_obs": (C.c_int32, [_vp]),
    "rf_model_describe": (C.c_int, [_vp, C.c_char_p, C.c_int32]),
    "rf_data_upload": (C.c_int, [_vp, C.POINTER(_vp), _ip, C.c_int64, _i64p, C.c_int32, C.c_int32, C.POINTER(_vp)]),
    "rf_data_destroy": (None, [_vp]),
    "rf_data_n_events": (C.c_int64, [_vp]),
    "rf_data_n_sets": (C.c_int32, [_vp]),
    "rf_data_read": (C.c_int, [_vp, C.c_int32, C.c_int64, C.c_int64, _dp]),
    "rf_data_offsets": (C.c_int, [_vp, _i64p]),
    "rf_nll": (C.c_int, [_vp, _vp, _dp, _dp, _vp]),
    "rf_nll_grad": (C.c_int, [_vp, _vp, _dp, _dp, _dp, _vp]),
    "rf_nll_grad_async": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "rf_nll_chunks": (C.c_int, [_vp, _vp, _dp, C.c_int32, _dp, C.c_int32, _ip]),
    "rf_model_set_fp64": (C.c_int, [_vp, C.c_int32]),
    "rf_set_launch": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "rf_autotune": (C.c_int, [_vp, _vp, C.c_int32, _ip, _ip, _dp]),
    "rf_autotune_scan": (C.c_int, [_vp, _vp, C.c_int32, C.c_int32, _ip, _dp, _ip]),
    "rf_fit": (C.c_int, [_vp, _vp, _dp, C.POINTER(rf_fit_opts), _dp, _dp, _dp, _ip, _ip]),
    "rf_fit_sets": (C.c_int, [_vp, _vp, _ip, C.c_int32, _dp, C.POINTER(rf_fit_opts), _dp, _dp, _dp, _ip, _ip]),
    "rf_generate_toys": (C.c_int, [_vp, _dp, C.c_int32, C.c_uint64, C.c_int32, _dp, C.c_int32, _ip, C.POINTER(_vp)]),
    "rf_hist64": (C.c_int, [_vp, _vp, C.c_int32, _vp, _vp]),
    "rf_data_refill": (C.c_int, [_vp, C.POINTER(_vp), _vp]),
    "rf_kernel_timing": (C.c_int, [C.c_int32]),
    "rf_kernel_time": (C.c_int, [_dp, _i64p, C.c_int32]),
    "rf_launch_count": (C.c_int, [_i64p]),
    "rf_slow_events": (C.c_int, [_vp, _i64p]),
    "rf_probe": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _dp]),
    "rf_nll_grad_noalloc": (C.c_int, [_vp, C.POINTER(_vp), _ip, C.c_int64, _vp, _vp, _vp, _vp]),
    "rf_nll_grad_noalloc_max_events": (C.c_int, [_vp, _i64p]),
    "rf_nll_grad_stream": (C.c_int, [_vp, _vp, C.POINTER(_vp), _dp, _dp, _dp, _vp]),
    "rf_binned_create": (C.c_int, [C.c_int32, C.c_int32, _ip, _ip, _dp, C.c_int32, _ip, C.c_int32, _vp, _dp,
                                   C.POINTER(_vp)]),
    "rf_binned_destroy": (None, [_vp]),
    "rf_binned_n_params": (C.c_int32, [_vp]),
    "rf_binned_nll_grad": (C.c_int, [_vp, C.c_int32, _dp, _dp, _dp, _dp]),
    "rf_binned_nll_grad_async": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, _vp, _vp]),
    "rf_binned_expected": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp]),
    "rf_binned_fit": (C.c_int, [_vp, C.c_int32, _dp, _dp, _dp, _dp, _vp, _dp, _dp, _dp, _ip, _ip]),
    "rf_shard": (C.c_int, [C.c_int64, C.c_int64, C.c_int32, C.c_int32, _i64p, _i64p]),
    "rf_nll_grad_partial": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "rf_combine_partials": (C.c_int, [_dp, _ip, C.c_int32, C.c_int32, C.c_int32, _dp, _ip]),
    "rf_mlp_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(_vp)]),
    "rf_mlp_destroy": (None, [_vp]),
    "rf_mlp_n_params": (C.c_int64, [_vp]),
    "rf_mlp_get_params": (C.c_int, [_vp, C.POINTER(C.c_float)]),
    "rf_mlp_set_params": (C.c_int, [_vp, C.POINTER(C.c_float)]),
    "rf_mlp_forward": (C.c_int, [_vp, _vp, C.c_int32, _vp, _vp]),
    "rf_mlp_predict": (C.c_int, [_vp, _vp, _vp, C.c_int32, _dp]),
    "rf_mlp_grad": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.POINTER(C.c_float), _vp, _vp]),
    "rf_mlp_adam": (C.c_int, [_vp, C.c_float, _vp]),
    "rf_mlp_train": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_uint64, C.c_int32,
                               C.POINTER(C.c_float)]),
    "rf_mlp_save": (C.c_int, [_vp, C.c_char_p]),
    "rf_mlp_load": (C.c_int, [C.c_char_p, C.POINTER(_vp)]),
    "rf_math_eval": (C.c_int, [C.c_int32, _vp, _vp, C.c_int64, _vp]),
    "rf_last_error": (C.c_char_p, []),
    "rf_version": (C.c_char_p, []),
}

_lib = None


class RFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load():
    """Load librfgpu.so (build it first with build.build()); raises if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2003_12861_gb300.build` "
                              "(the CUDA library is required; there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, allow=(RF_OK,)) -> int:
    if status not in allow:
        raise RFError(status, load().rf_last_error().decode())
    return status
