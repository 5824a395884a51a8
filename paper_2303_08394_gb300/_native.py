"""ctypes declarations for libkifmm.so (include/kifmm.h).

Loading fails loudly when the shared library is missing: there is no CPU
fallback.  Build it with ``python -m paper_2303_08394_gb300.build``.
"""
from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libkifmm.so")

FMM_OK, FMM_ERR_INVALID_ARG, FMM_ERR_CUDA, FMM_ERR_OOM, FMM_ERR_TIMEOUT, \
    FMM_ERR_UNSUPPORTED = range(6)
STATUS_NAMES = {0: "FMM_OK", 1: "FMM_ERR_INVALID_ARG", 2: "FMM_ERR_CUDA",
                3: "FMM_ERR_OOM", 4: "FMM_ERR_TIMEOUT", 5: "FMM_ERR_UNSUPPORTED"}
M2L_FP32, M2L_BF16X3, M2L_TF32X3 = 0, 1, 2
OPT_M2L_MODE = 1
OPT_GRAPH = 2
OPT_AUTOTUNE = 3
OPT_GEMM_SHAPE = 4
OPT_TEST_M2L_STALL = 5
OPT_M2L_KERNEL = 6
OPT_FORCE_KNOBS = 7
TREE_AUTO, TREE_HOST, TREE_DEVICE, TREE_LEVELS_HOST = 0, 1, 2, 3

INFO = {"n": 0, "nodes": 1, "leaves": 2, "depth": 3, "nsurf": 4, "rank_m2l": 5,
        "rank_up": 6, "rank_down": 7, "u_pairs": 8, "v_pairs": 9, "w_pairs": 10,
        "x_pairs": 11, "p2p_pairs": 12, "m2l_tiles": 13, "m2l_entries": 14,
        "last_launches": 15, "points": 16, "problems": 17, "device_trees": 18, "operator_source": 19,
        "m2l_windows": 20, "m2l_items": 21, "m2l_kernel": 22, "tunings": 23,
        "surf_pairs": 24, "wx_direct_pairs": 25}
ARRAYS = {"node_keys": (0, "i4"), "node_range": (1, "i8"), "leaf_flag": (2, "i4"),
          "perm": (3, "i8"), "u_ptr": (4, "i8"), "u_idx": (5, "i4"),
          "v_ptr": (6, "i8"), "v_idx": (7, "i4"), "w_ptr": (8, "i8"),
          "w_idx": (9, "i4"), "x_ptr": (10, "i8"), "x_idx": (11, "i4"),
          "surface": (12, "f8"), "m2l_u": (13, "f8"), "m2l_v": (14, "f8"),
          "m2l_s": (15, "f8"), "root": (16, "f8"), "charge_row": (17, "i8"),
          "output_row": (18, "i8"), "node_problem": (19, "i4"), "gemm_shapes": (20, "i4"),
          "m2l_tile_level": (21, "i4"), "m2l_tile_target": (22, "i4"),
          "m2l_tile_entry_ptr": (23, "i4"), "m2l_entry_offset": (24, "i4"),
          "m2l_entry_src": (25, "i4"), "op_pu": (26, "f8"), "op_ps": (27, "f8"),
          "op_pv": (28, "f8"), "op_qu": (29, "f8"), "op_qs": (30, "f8"), "op_qv": (31, "f8"),
          "op_m2m": (32, "f8"), "op_l2l": (33, "f8"), "op_quk": (34, "f8"),
          "m2l_win_target_ptr": (35, "i4"), "m2l_win_targets": (36, "i4"),
          "m2l_win_item_ptr": (37, "i4"), "m2l_item_offset": (38, "i4"),
          "m2l_item_pair_ptr": (39, "i4"), "m2l_pair_src": (40, "i4"),
          "m2l_pair_slot": (41, "i4"), "m2l_cta_ptr": (42, "i4"), "m2l_cta_win": (43, "i4"),
          "m2l_tile_cta_ptr": (44, "i4"), "m2l_tile_cta_tiles": (45, "i4"),
          "tuned_knobs": (46, "i4")}

# every symbol include/kifmm.h declares
EXPORTS = ("fmm_options_init", "fmm_plan_create", "fmm_plan_create_ex",
           "fmm_plan_create_batch", "fmm_plan_create_batch_ex", "fmm_set_operator_cache", "fmm_plan_set_option", "fmm_evaluate", "fmm_evaluate_gradient", "fmm_evaluate_noalloc", "fmm_destroy",
           "fmm_last_error", "fmm_plan_info", "fmm_plan_get_array", "fmm_plan_get_workspace", "fmm_plan_phase_ms")


class Options(ctypes.Structure):
    _fields_ = [("alpha_inner", ctypes.c_double), ("alpha_outer", ctypes.c_double),
                ("rcond", ctypes.c_double), ("eps_svd", ctypes.c_double),
                ("max_level", ctypes.c_int32), ("balance", ctypes.c_int32),
                ("m2l_mode", ctypes.c_int32), ("host_only", ctypes.c_int32),
                ("device", ctypes.c_int32), ("tree_build", ctypes.c_int32),
                ("direct_wx", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class FMMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FileNotFoundError(
            f"{LIB_PATH} is missing; build it with python -m paper_2303_08394_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, dp, fp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
    L.fmm_options_init.argtypes = [ctypes.POINTER(Options)]
    L.fmm_options_init.restype = None
    L.fmm_plan_create.argtypes = [dp, dp, i64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
    L.fmm_plan_create_ex.argtypes = [dp, dp, i64, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(Options), ctypes.POINTER(vp)]
    pp = ctypes.POINTER(ctypes.c_void_p)
    L.fmm_plan_create_batch.argtypes = [pp, pp, ctypes.POINTER(i64), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(vp)]
    L.fmm_plan_create_batch_ex.argtypes = [pp, pp, ctypes.POINTER(i64), ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.POINTER(Options),
                                           ctypes.POINTER(vp)]
    L.fmm_plan_set_option.argtypes = [vp, ctypes.c_int, ctypes.c_double]
    L.fmm_set_operator_cache.argtypes = [ctypes.c_char_p]
    L.fmm_evaluate.argtypes = [vp, fp, ctypes.c_int, dp, vp]
    L.fmm_evaluate_noalloc.argtypes = [vp, fp, ctypes.c_int, dp, vp]
    L.fmm_evaluate_gradient.argtypes = [vp, fp, ctypes.c_int, dp, dp, vp]
    L.fmm_destroy.argtypes = [vp]
    L.fmm_destroy.restype = None
    L.fmm_last_error.argtypes = []
    L.fmm_last_error.restype = ctypes.c_char_p
    L.fmm_plan_info.argtypes = [vp, ctypes.c_int, ctypes.POINTER(i64)]
    L.fmm_plan_get_array.argtypes = [vp, ctypes.c_int, vp, i64, ctypes.POINTER(i64)]
    L.fmm_plan_get_workspace.argtypes = [vp, ctypes.c_int, vp, i64, ctypes.POINTER(i64)]
    L.fmm_plan_phase_ms.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    for name in ("fmm_plan_create", "fmm_plan_create_ex", "fmm_plan_create_batch",
                 "fmm_plan_create_batch_ex", "fmm_plan_set_option",
                 "fmm_evaluate", "fmm_evaluate_gradient", "fmm_evaluate_noalloc", "fmm_plan_info", "fmm_plan_get_array", "fmm_plan_phase_ms"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(status):
    if status != FMM_OK:
        raise FMMError(status, lib().fmm_last_error().decode(errors="replace"))
