"""ctypes declarations of the C ABI in include/scuc_lp.h (marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "libscuclp.so")

SCUC_OK, SCUC_E_INVALID, SCUC_E_CUDA, SCUC_E_OOM, SCUC_E_DEVICE_TIMEOUT, SCUC_E_INFEASIBLE = range(6)
STATUS = {0: "optimal", 1: "iter_limit", 2: "time_limit", 3: "numerical", 4: "fallback_cold",
          5: "primal_infeasible", 6: "dual_infeasible"}
ALGO = {"hpr": 0, "pdhg_avg": 1}
FP64, MIXED = 0, 1


class SolveParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int64), ("time_limit_s", C.c_double),
                ("check_every", C.c_int32), ("precision", C.c_int32), ("use_scaling", C.c_int32),
                ("sigma0", C.c_double), ("lambda_in", C.c_double), ("lambda_safety", C.c_double),
                ("power_max_iter", C.c_int32), ("power_tol", C.c_double), ("power_seed", C.c_uint64),
                ("restart_suff", C.c_double), ("restart_nec", C.c_double),
                ("restart_long", C.c_double), ("polish_factor", C.c_double),
                ("polish_stall", C.c_int32), ("use_graph", C.c_int32), ("profile", C.c_int32),
                ("device_ptrs", C.c_int32), ("restart_ref", C.c_int32),
                ("restart_metric", C.c_int32), ("sigma_update", C.c_int32), ("algo", C.c_int32),
                ("infeas_tol", C.c_double), ("spmv_layout", C.c_int32), ("split_steps", C.c_int32),
                ("polish_floor", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("restarts", C.c_int32), ("iters", C.c_int64),
                ("iters_fp32", C.c_int64), ("power_iters", C.c_int32), ("nlog", C.c_int32),
                ("kkt", C.c_double), ("rp", C.c_double), ("rd", C.c_double), ("gap", C.c_double),
                ("pobj", C.c_double), ("dobj", C.c_double), ("lambda_", C.c_double),
                ("sigma", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("ms_dual_spmv", C.c_double),
                ("ms_primal_spmv", C.c_double), ("n_dual_spmv", C.c_int64),
                ("n_primal_spmv", C.c_int64), ("ms_dual_spmv_f32", C.c_double),
                ("ms_primal_spmv_f32", C.c_double), ("n_dual_spmv_f32", C.c_int64),
                ("n_primal_spmv_f32", C.c_int64), ("launches", C.c_int64),
                ("warm_iters", C.c_int64), ("ref_iters", C.c_int64), ("cold_first_kkt", C.c_double)]


class BatchInfo(C.Structure):
    _fields_ = [("autotune", C.c_int32), ("ept_A", C.c_int32), ("run_A", C.c_int32), ("ept_T", C.c_int32),
                ("run_T", C.c_int32), ("candidates", C.c_int32), ("blocks_A", C.c_int32),
                ("blocks_T", C.c_int32), ("setup_ms", C.c_double), ("tune_ms", C.c_double),
                ("solve_ms", C.c_double), ("total_ms", C.c_double), ("launches", C.c_int64),
                ("periods", C.c_int64), ("scale_ms", C.c_double), ("tune_cached", C.c_int32),
                ("reserved0", C.c_int32)]


class CheckLog(C.Structure):
    _fields_ = [("iter", C.c_int64), ("restart", C.c_int32), ("first", C.c_int32),
                ("rp", C.c_double), ("rd", C.c_double), ("gap", C.c_double), ("pobj", C.c_double),
                ("dobj", C.c_double), ("rho", C.c_double), ("sigma", C.c_double),
                ("fp64", C.c_int32), ("pad", C.c_int32)]


class ScucMap(C.Structure):
    _fields_ = [("G", C.c_int32), ("T", C.c_int32), ("u_idx", C.c_void_p), ("v_idx", C.c_void_p),
                ("w_idx", C.c_void_p), ("u_init", C.c_void_p)]


class FixParams(C.Structure):
    _fields_ = [("tau", C.c_double), ("t_first", C.c_int32), ("max_passes", C.c_int32),
                ("x_on_device", C.c_int32), ("build_reduced", C.c_int32)]


class FixInfo(C.Structure):
    _fields_ = [("nfixed", C.c_int64), ("passes", C.c_int32), ("infeasible", C.c_int32),
                ("m_red", C.c_int32), ("n_red", C.c_int32), ("nnz_red", C.c_int64),
                ("n_fixed_cols", C.c_int64), ("obj_const", C.c_double), ("ms", C.c_double),
                ("ms_propagate", C.c_double), ("ms_reduce", C.c_double), ("ms_setup", C.c_double)]


class WsTrainParams(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("w_dispatch", C.c_float), ("w_price", C.c_float)]


class WsLayout(C.Structure):
    _fields_ = [("G", C.c_int32), ("T", C.c_int32), ("nseg", C.c_int32), ("fill", C.c_int32),
                ("u_col", C.c_void_p), ("v_col", C.c_void_p), ("w_col", C.c_void_p),
                ("p_col", C.c_void_p), ("seg_col", C.c_void_p), ("p_cap", C.c_void_p),
                ("seg_cap", C.c_void_p), ("u_init", C.c_void_p), ("unit_price_row", C.c_void_p),
                ("nprice", C.c_int32), ("price_row", C.c_void_p), ("price_ptr", C.c_void_p),
                ("price_member", C.c_void_p), ("price_scale", C.c_double)]


class WarmParams(C.Structure):
    _fields_ = [("warm_max_iter", C.c_int64), ("first_check", C.c_int32), ("cold_first_kkt", C.c_double)]


WS_FILL_VW, WS_FILL_SEGMENTS, WS_FILL_PRICES = 1, 2, 4

_lib = None

# exported symbols and their signatures
_SIGS = {
    "scuc_default_params": (None, [C.POINTER(SolveParams)]),
    "scuc_lp_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.c_int64, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "scuc_lp_create_box": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.c_int64,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "scuc_lp_dims": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int64)]),
    "scuc_lp_layout": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "scuc_lp_set_index16": (C.c_int, [C.c_void_p, C.c_int32]),
    "scuc_lp_solve": (C.c_int, [C.c_void_p, C.POINTER(SolveParams), C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveInfo)]),
    "scuc_lp_get_log": (C.c_int, [C.c_void_p, C.POINTER(CheckLog), C.c_int32, C.POINTER(C.c_int32)]),
    "scuc_lp_matvec": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "scuc_lp_solve_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(SolveParams),
                                      C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                      C.POINTER(SolveInfo), C.POINTER(BatchInfo)]),
    "scuc_lp_kkt_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "scuc_probe_fma_peak": (C.c_int, [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "scuc_ws_set_gemm": (C.c_int, [C.c_void_p, C.c_int32]),
    "scuc_default_fix_params": (None, [C.POINTER(FixParams)]),
    "scuc_fix_and_propagate": (C.c_int, [C.c_void_p, C.POINTER(ScucMap), C.c_void_p, C.c_void_p,
                                         C.POINTER(FixParams), C.c_void_p, C.POINTER(C.c_void_p),
                                         C.c_void_p, C.c_void_p, C.POINTER(FixInfo)]),
    "scuc_lp_get_bounds": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "scuc_lp_set_bounds": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "scuc_lp_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "scuc_lp_row_violations": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.c_int32,
                                         C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "scuc_lp_add_rows": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "scuc_lp_destroy": (None, [C.c_void_p]),
    "scuc_ws_default_train_params": (None, [C.POINTER(WsTrainParams)]),
    "scuc_ws_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.c_void_p]),
    "scuc_ws_num_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "scuc_ws_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "scuc_ws_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "scuc_ws_set_input_norm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "scuc_ws_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "scuc_ws_gradients": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                    C.POINTER(WsTrainParams), C.c_void_p, C.POINTER(C.c_double)]),
    "scuc_ws_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32,
                                C.c_int32, C.POINTER(WsTrainParams), C.c_void_p]),
    "scuc_ws_destroy": (None, [C.c_void_p]),
    "scuc_ws_assemble": (C.c_int, [C.c_void_p, C.POINTER(WsLayout), C.c_void_p, C.c_void_p, C.c_void_p]),
    "scuc_ws_targets": (C.c_int, [C.c_void_p, C.POINTER(WsLayout), C.c_void_p, C.c_void_p, C.c_void_p]),
    "scuc_default_warm_params": (None, [C.POINTER(WarmParams)]),
    "scuc_lp_solve_warm": (C.c_int, [C.c_void_p, C.POINTER(SolveParams), C.c_void_p, C.c_void_p,
                                     C.POINTER(WarmParams), C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.POINTER(SolveInfo)]),
    "scuc_last_error": (C.c_char_p, []),
}


def lib():
    """Load the in-tree library; raise if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(SO):
            raise RuntimeError("libscuclp.so is missing: build it with "
                               "`python -m paper_2510_10891_b300.build` (nvcc, sm_103a)")
        L = C.CDLL(SO)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class ScucError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("scuc error %d: %s" % (code, msg))
        self.code = code


def check(rc):
    if rc != SCUC_OK:
        raise ScucError(rc, lib().scuc_last_error().decode(errors="replace"))
    return rc
