"""ctypes binding of libqcs.so (include/qcs.h): argument marshalling only.

The library is built in-tree by ``paper_2303_08989_gb300.build`` into
``paper_2303_08989_gb300/_build/libqcs.so``.  Loading fails loudly when it is
missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libqcs.so")

QCS_SUCCESS = 0
QCS_ERR_INVALID_ARG = -1
QCS_ERR_UNSUPPORTED = -2
QCS_ERR_ALLOC = -3
QCS_ERR_CUDA = -4
QCS_ERR_TIMEOUT = -5
QCS_ERR_SCRATCH_TOO_SMALL = -6

MODE_AUTO, MODE_FP16X, MODE_FP16X_SCALED, MODE_TF32X, MODE_FP32, MODE_BF16X3 = range(6)
MODE_BY_NAME = {"auto": 0, "fp16x": 1, "fp16x_scaled": 2, "tf32x": 3, "fp32": 4, "bf16x3": 5}
MODE_NAME = {v: k for k, v in MODE_BY_NAME.items()}
MODE_FP16X_ROWCOL = 6  # reported only, never an argument (qcs_set_rowcol_scaling)
MODE_NAME[MODE_FP16X_ROWCOL] = "fp16x_rowcol"
OP_N, OP_T, OP_C = 0, 1, 2

#: every entry point include/qcs.h declares
EXPORTED = [
    "qcs_create", "qcs_destroy", "qcs_set_stream", "qcs_set_underflow_tol", "qcs_set_size_rule",
    "qcs_set_drain_stages",
    "qcs_exp_stats", "qcs_select", "qcs_cgemm", "qcs_split", "qcs_permute", "qcs_contract_tree",
    "qcs_contract_tree_backward", "qcs_set_profiling", "qcs_get_profile", "qcs_sync",
    "qcs_status_string", "qcs_cgemm_noalloc", "qcs_tree_graph_create", "qcs_tree_graph_launch",
    "qcs_tree_graph_destroy", "qcs_get_auto_counts", "qcs_autotune_gemm", "qcs_autotune_tree",
    "qcs_get_tuning", "qcs_set_tuning", "qcs_set_instance_batch", "qcs_set_tc_schedule",
    "qcs_set_tc_splits", "qcs_sgemm", "qcs_set_complex_products", "qcs_set_wait_budget",
    "qcs_debug_stall_producer", "qcs_cgemm_noalloc_status", "qcs_measure_fma_peak",
    "qcs_set_fused_split", "qcs_set_tree_levels", "qcs_set_group_budget", "qcs_fidelity_stats",
    "qcs_tree_layout_info", "qcs_set_tc_multicast", "qcs_set_tc_pairs",
    "qcs_selection_stats", "qcs_tree_backward_graph_create", "qcs_set_rowcol_scaling",
    "qcs_rowcol_stats",
]
SIZE_RULE_OFF, SIZE_RULE_PAPER, SIZE_RULE_TUNED = 0, 1, 2
NUM_MODES = 6
PROFILE_STAGES = ["stats", "select", "split", "gemm_tc", "gemm_simt", "permute", "reduce"]


class QcsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})" if what else status_string(code))


class qcs_c32(ctypes.Structure):
    _fields_ = [("x", ctypes.c_float), ("y", ctypes.c_float)]


class qcs_stats_t(ctypes.Structure):
    _fields_ = [("hist", ctypes.c_int64 * 256), ("n_zero", ctypes.c_int64), ("n", ctypes.c_int64)]


class qcs_gemm_desc_t(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("sA", ctypes.c_int32), ("sB", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


MAX_RANK = 32


class qcs_selection_stats_t(ctypes.Structure):
    _fields_ = [("e_max", ctypes.c_int32), ("stage2", ctypes.c_int32),
                ("n_nonzero", ctypes.c_int64), ("n_nonfinite", ctypes.c_int64),
                ("n_under_fp16", ctypes.c_int64), ("n_under_window", ctypes.c_int64)]


class qcs_tune_entry_t(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("opA", ctypes.c_int32), ("opB", ctypes.c_int32),
                ("ms", ctypes.c_float * 6), ("best", ctypes.c_int32), ("reps", ctypes.c_int32),
                ("splits", ctypes.c_int32), ("group_m", ctypes.c_int32)]


class qcs_gather_t(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("dims", ctypes.c_int64 * MAX_RANK), ("strides", ctypes.c_int64 * MAX_RANK)]


class qcs_step_t(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int32), ("b", ctypes.c_int32), ("direct_a", ctypes.c_int32),
                ("direct_b", ctypes.c_int32), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("k", ctypes.c_int64), ("map_a", qcs_gather_t), ("map_b", qcs_gather_t),
                ("mode", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class qcs_tree_t(ctypes.Structure):
    _fields_ = [("n_leaves", ctypes.c_int32), ("n_steps", ctypes.c_int32),
                ("n_instances", ctypes.c_int32), ("n_slots", ctypes.c_int32),
                ("leaf_size", ctypes.POINTER(ctypes.c_int64)),
                ("instance_offset", ctypes.POINTER(ctypes.c_int64)),
                ("instance_slot", ctypes.POINTER(ctypes.c_int32)),
                ("steps", ctypes.POINTER(qcs_step_t)), ("out_size", ctypes.c_int64),
                ("out_index", ctypes.POINTER(ctypes.c_int64))]


class qcs_run_info_t(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double), ("gemm_count", ctypes.c_int64),
                ("gather_count", ctypes.c_int64), ("mode_count", ctypes.c_int64 * 6),
                ("workspace_bytes", ctypes.c_int64), ("flops", ctypes.c_double),
                ("mode_flops", ctypes.c_double * 6), ("level_launches", ctypes.c_int64),
                ("level_gemms", ctypes.c_int64)]


class qcs_tree_layout_t(ctypes.Structure):
    _fields_ = [("total_bytes", ctypes.c_int64), ("group", ctypes.c_int32),
                ("batched_steps", ctypes.c_int32), ("level_launches", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libqcs.so and declare every prototype.  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    I64 = ctypes.c_int64
    H = ctypes.c_void_p
    sig = {
        "qcs_create": [ctypes.POINTER(ctypes.c_void_p), P],
        "qcs_destroy": [H],
        "qcs_set_stream": [H, P],
        "qcs_set_underflow_tol": [H, ctypes.c_double],
        "qcs_set_size_rule": [H, I],
        "qcs_set_drain_stages": [H, I],
        "qcs_exp_stats": [H, I64, I64, P, I64, P],
        "qcs_select": [H, P, P, P],
        "qcs_cgemm": [H, I, I, I, I64, I64, I64, ctypes.POINTER(qcs_c32), P, I64, P, I64,
                      ctypes.POINTER(qcs_c32), P, I64, P],
        "qcs_sgemm": [H, I, I, I, I64, I64, I64, ctypes.POINTER(ctypes.c_float), P, I64, P, I64,
                      ctypes.POINTER(ctypes.c_float), P, I64, P],
        "qcs_split": [H, P, I, I, I64, I64, P, I64, P, I64, I64],
        "qcs_permute": [H, I, ctypes.POINTER(I64), ctypes.POINTER(I64), I64, P, P, P],
        "qcs_contract_tree": [H, ctypes.POINTER(qcs_tree_t), ctypes.POINTER(P), P,
                              ctypes.POINTER(qcs_run_info_t)],
        "qcs_contract_tree_backward": [H, ctypes.POINTER(qcs_tree_t), ctypes.POINTER(P), P,
                                       ctypes.POINTER(P), ctypes.POINTER(qcs_run_info_t)],
        "qcs_set_profiling": [H, I],
        "qcs_get_profile": [H, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64), I],
        "qcs_sync": [H],
        "qcs_cgemm_noalloc": [P, I, ctypes.c_double, I, I, I64, I64, I64, ctypes.POINTER(qcs_c32),
                              P, I64, P, I64, ctypes.POINTER(qcs_c32), P, I64, P],
        "qcs_tree_graph_create": [H, ctypes.POINTER(qcs_tree_t), ctypes.POINTER(P), P,
                                  ctypes.POINTER(ctypes.c_void_p)],
        "qcs_tree_backward_graph_create": [H, ctypes.POINTER(qcs_tree_t), ctypes.POINTER(P), P,
                                           ctypes.POINTER(P), ctypes.POINTER(ctypes.c_void_p)],
        "qcs_tree_graph_launch": [P],
        "qcs_tree_graph_destroy": [P],
        "qcs_get_auto_counts": [H, ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_double), I],
        "qcs_autotune_gemm": [H, I, I, I64, I64, I64, I, ctypes.POINTER(qcs_tune_entry_t)],
        "qcs_autotune_tree": [H, ctypes.POINTER(qcs_tree_t), I, I, ctypes.POINTER(I64)],
        "qcs_get_tuning": [H, ctypes.POINTER(qcs_tune_entry_t), I64, ctypes.POINTER(I64)],
        "qcs_set_tuning": [H, ctypes.POINTER(qcs_tune_entry_t), I64],
        "qcs_set_instance_batch": [H, I],
        "qcs_set_tc_schedule": [H, I, I],
        "qcs_set_tc_splits": [H, I],
        "qcs_set_complex_products": [H, I],
        "qcs_set_wait_budget": [H, ctypes.c_uint64],
        "qcs_debug_stall_producer": [H, I],
        "qcs_cgemm_noalloc_status": [P, I],
        "qcs_measure_fma_peak": [H, ctypes.POINTER(ctypes.c_double)],
        "qcs_set_fused_split": [H, I],
        "qcs_set_tree_levels": [H, I],
        "qcs_set_tc_multicast": [H, I],
        "qcs_set_tc_pairs": [H, I],
        "qcs_set_rowcol_scaling": [H, I],
        "qcs_rowcol_stats": [H, I, I, I64, I64, I64, P, I64, P, I64, P, P, P],
        "qcs_set_group_budget": [H, ctypes.c_uint64],
        "qcs_fidelity_stats": [H, P, I, P, I64, P],
        "qcs_tree_layout_info": [ctypes.POINTER(qcs_tree_t), I, I, I, I, ctypes.c_uint64, P, P,
                                 P, P, P, ctypes.POINTER(qcs_tree_layout_t)],
        "qcs_selection_stats": [H, I, I, I64, I64, I64, P, I64, P, I64,
                                ctypes.POINTER(qcs_selection_stats_t), ctypes.POINTER(qcs_gemm_desc_t)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = I
    lib.qcs_status_string.argtypes = [I]
    lib.qcs_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().qcs_status_string(code).decode()
    except ImportError:
        return f"status {code}"


def check(code: int, what: str = ""):
    if code != QCS_SUCCESS:
        raise QcsError(code, what)
    return code
