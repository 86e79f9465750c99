"""ctypes declarations of the C ABI in include/ue.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libue.so")

UE_OK = 0
UE_ERR_ARG = -1
UE_ERR = {-1: "UE_ERR_ARG", -2: "UE_ERR_NONMANIFOLD", -3: "UE_ERR_DEGENERATE", -4: "UE_ERR_DUAL",
          -5: "UE_ERR_CUDA", -6: "UE_ERR_ALLOC", -7: "UE_ERR_UNSTABLE", -8: "UE_ERR_TIMEOUT"}
UE_REORDER_NONE, UE_REORDER_RCM, UE_REORDER_KD, UE_REORDER_GREEDY, UE_REORDER_GREEDY_RINGS = 0, 1, 2, 3, 4
UE_PREC_FP32, UE_PREC_FP64 = 0, 1
UE_DT_GIVEN, UE_DT_POWER, UE_DT_LEARNED = 0, 1, 2
UE_RHO_GIVEN, UE_RHO_POWER, UE_RHO_LEARNED, UE_RHO_POWER_FALLBACK = 0, 1, 2, 3
UE_MLP_PARAMS = 5057
UE_VARIANT_PLAIN, UE_VARIANT_BLOCKED, UE_VARIANT_PERSISTENT = 1, 2, 3
UE_TB_SPLIT, UE_TB_FUSED = 0, 1
UE_STATIC_MAX_TRIS, UE_STATIC_MAX_EDGES = 1 << 18, 1 << 19

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("reorder", C.c_int32), ("precision", C.c_int32), ("dt_mode", C.c_int32),
                ("power_iters", C.c_int32), ("power_seed", C.c_uint32), ("variant", C.c_int32),
                ("graph_chunk", C.c_int32), ("tile_tris", C.c_int32), ("block_depth", C.c_int32),
                ("tb_threads", C.c_int32), ("dt", C.c_double),
                ("safety", C.c_double), ("watchdog_growth", C.c_double),
                ("watchdog_every", C.c_int32), ("tb_kernel", C.c_int32),
                ("mlp_params", C.c_void_p), ("learned_margin", C.c_double),
                ("timeout_ms", C.c_int32), ("test_skip_cta", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tris", C.c_int64), ("n_edges", C.c_int64),
                ("n_interior_edges", C.c_int64), ("steps_done", C.c_int64), ("dt", C.c_double),
                ("rho", C.c_double), ("rho_source", C.c_int32), ("precision", C.c_int32),
                ("bytes_per_step", C.c_double), ("kernel_launches", C.c_int64),
                ("dt_setup_ms", C.c_double), ("rho_lo", C.c_double), ("rho_hi", C.c_double),
                ("rho_hat", C.c_double), ("direct_fields", C.c_int64), ("tb_kernel_used", C.c_int32),
                ("reserved2", C.c_int32)]


P = C.c_void_p
I64 = C.c_int64
PD = C.POINTER(C.c_double)
PI32 = C.POINTER(C.c_int32)
PI64 = C.POINTER(C.c_int64)

# (name, restype, argtypes) for every exported entry point of include/ue.h
SIGNATURES = [
    ("ue_options_default", None, [C.POINTER(Options)]),
    ("ue_mesh_load", C.c_int, [PD, I64, PI32, I64, C.POINTER(Options), ALLOC_FN, FREE_FN, P, C.POINTER(P)]),
    ("ue_geometry_build", C.c_int, [P, C.POINTER(Options), P]),
    ("ue_batch_create", C.c_int, [C.POINTER(P), C.c_int32, P, C.POINTER(P)]),
    ("ue_get_dt", C.c_int, [P, PD, PD, PI32]),
    ("ue_set_plasma", C.c_int, [P, PD, C.c_double]),
    ("ue_set_source", C.c_int, [P, PI32, PD, I64, C.c_double, C.c_double, C.c_double]),
    ("ue_write_fields", C.c_int, [P, PD, PD, PD, P]),
    ("ue_write_fields_f32", C.c_int, [P, P, P, P, P]),
    ("ue_read_fields_f32", C.c_int, [P, P, P, P, P]),
    ("ue_step_n", C.c_int, [P, I64, P]),
    ("ue_step_prepare", C.c_int, [P, P]),
    ("ue_exchange_tris", C.c_int, [P, P, I64, P, C.c_int32, P]),
    ("ue_read_fields", C.c_int, [P, PD, PD, PD, P]),
    ("ue_energy", C.c_int, [P, PD, P]),
    ("ue_check", C.c_int, [P, PD, PI32]),
    ("ue_get_step", C.c_int, [P, PI64]),
    ("ue_set_step", C.c_int, [P, I64]),
    ("ue_get_sizes", C.c_int, [P, PI64, PI64, PI64, PI64]),
    ("ue_get_tables", C.c_int, [P, PI64, PI64, PI32, PI32]),
    ("ue_get_tiles", C.c_int, [P, PI64, PI64]),
    ("ue_frame_attach", C.c_int, [P, C.c_int32, C.c_double, C.c_int32]),
    ("ue_frame_get", C.c_int, [P, PI64, PD]),
    ("ue_frame_interface", C.c_int, [P, PI64, PI64]),
    ("ue_frame_region", C.c_int, [P, C.c_int32, PI64]),
    ("ue_frame_state", C.c_int, [P, PD, PD, PD, PD, C.c_int32, P]),
    ("ue_frame_fields", C.c_int, [P, PD, PD, PD, P]),
    ("ue_get_geometry", C.c_int, [P, PD, PD, PD, PD]),
    ("ue_rho_features", C.c_int, [P, P, P, P]),
    ("ue_mlp_forward", C.c_int, [P, P, I64, C.c_int32, P, P]),
    ("ue_mlp_backward", C.c_int, [P, P, P, P, I64, C.c_int32, P, P, P]),
    ("ue_adam", C.c_int, [P, P, P, P, C.c_int32, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int32, P]),
    ("ue_seg_argmax", C.c_int, [P, P, P, C.c_int32, P, P, P]),
    ("ue_rho_loss", C.c_int, [P, P, C.c_int32, P, P, P]),
    ("ue_profile_steps", C.c_int, [P, I64, P, PD, PD]),
    ("ue_power_iteration_static", C.c_int, [P, P, P, P, P, P, I64, I64, C.c_int32, C.c_uint32, P, PD]),
    ("ue_modes", C.c_int, [P, C.c_int32, C.c_int32, C.c_uint32, PD, PD, P]),
    ("ue_modes_low", C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, C.c_uint32, PD, PD, P]),
    ("ue_mesh_relax", C.c_int, [PD, I64, PI32, I64, PD, C.c_int32, C.c_int32, C.c_double, PI32, I64,
                                PI32, I64, PD, PI32, PI64, P]),
    ("ue_mesh_flip", C.c_int, [PD, I64, PI32, I64, PI32, I64, PI32, PI64]),
    ("ue_triangulate", C.c_int, [PD, I64, PI32, I64, PD, I64, C.c_int32, PI32, I64, PI64, PI64]),
    ("ue_stats", C.c_int, [P, C.POINTER(Stats)]),
    ("ue_last_error", C.c_char_p, []),
    ("ue_mesh_free", None, [P]),
]

_lib = None


def lib():
    """Load libue.so (built in-tree); raise if it is missing: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1812_01448_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class UEError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().ue_last_error().decode(errors="replace")
        super().__init__(f"{where}: {UE_ERR.get(code, code)}: {msg}")
        self.code = code


def check(rc: int, where: str):
    if rc != UE_OK:
        raise UEError(rc, where)
