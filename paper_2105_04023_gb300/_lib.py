"""ctypes declarations of the C ABI in include/im.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libim.so")

IM_OK, IM_EINVAL, IM_ENOMEM, IM_ECUDA, IM_ETIMEOUT, IM_ECANCELED, IM_ENOTREADY = range(7)
STATUS_NAMES = {0: "IM_OK", 1: "IM_EINVAL", 2: "IM_ENOMEM", 3: "IM_ECUDA", 4: "IM_ETIMEOUT", 5: "IM_ECANCELED",
                6: "IM_ENOTREADY"}
IM_IC_CONST, IM_WC, IM_PER_EDGE = 0, 1, 2
IM_MEM_DEVICE, IM_MEM_HOST = 0, 1
IM_BLOCK_RESIDUAL, IM_BLOCK_LITERAL = 0, 1


class im_graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("xadj", ctypes.c_void_p), ("adj", ctypes.c_void_p),
                ("model", ctypes.c_int), ("p", ctypes.c_double), ("p_edge", ctypes.c_void_p),
                ("memory", ctypes.c_int), ("undirected", ctypes.c_int32)]


class im_params(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("K", ctypes.c_int32), ("eps_g", ctypes.c_double), ("eps_l", ctypes.c_double),
                ("eps_c", ctypes.c_double), ("seed", ctypes.c_uint64), ("max_sweeps", ctypes.c_int64),
                ("blocking", ctypes.c_int32)]


class im_trace(ctypes.Structure):
    _fields_ = [("seeds", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("estimate", ctypes.c_void_p),
                ("gsum", ctypes.c_void_p), ("rebuilt", ctypes.c_void_p)]


class im_stats(ctypes.Structure):
    _fields_ = [("visits", ctypes.c_uint64), ("prop_bytes", ctypes.c_uint64), ("sweeps", ctypes.c_int64),
                ("builds", ctypes.c_int64), ("bfs_levels", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("prop_launches", ctypes.c_int64), ("prop_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("sweep_ms", ctypes.c_double), ("scan_ms", ctypes.c_double), ("bfs_ms", ctypes.c_double),
                ("init_ms", ctypes.c_double), ("live_pairs", ctypes.c_uint64), ("first_bytes", ctypes.c_uint64),
                ("first_ms", ctypes.c_double), ("first_launches", ctypes.c_int64)]


class im_tuning(ctypes.Structure):
    _fields_ = [("first_sweep_blocks", ctypes.c_int32), ("stream_push", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("degree_class", ctypes.c_int32), ("best_ms", ctypes.c_double),
                ("default_ms", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64

SIGNATURES = {
    "im_ctx_create": (_I, [_I, _P, ctypes.POINTER(_P)]),
    "im_ctx_destroy": (_I, [_P]),
    "im_last_error": (ctypes.c_char_p, [_P]),
    "im_ctx_set_timing": (_I, [_P, _I]),
    "im_autotune": (_I, [_P, ctypes.POINTER(im_graph), ctypes.POINTER(im_params), ctypes.POINTER(im_tuning)]),
    "im_ctx_stats": (_I, [_P, ctypes.POINTER(im_stats)]),
    "im_build_sketches": (_I, [_P, ctypes.POINTER(im_graph), ctypes.POINTER(im_params), ctypes.POINTER(_P)]),
    "im_estimate": (_I, [_P, _P, _P, _I32, _P, _P]),
    "im_sketch_registers": (_I, [_P, _P, _P]),
    "im_sketch_info": (_I, [_P, _P, _P, _P, _P, _I64]),
    "im_sketch_destroy": (_I, [_P]),
    "im_sketch_export": (_I, [_P, _P, _P, ctypes.c_uint64, _P]),
    "im_sketch_import": (_I, [_P, ctypes.POINTER(im_graph), _P, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "im_select_seeds_from": (_I, [_P, _P, ctypes.POINTER(im_params), _P, _P, _P, ctypes.POINTER(im_trace)]),
    "im_select_seeds": (_I, [_P, ctypes.POINTER(im_graph), ctypes.POINTER(im_params), _P, _P, _P,
                             ctypes.POINTER(im_trace)]),
    "im_select_seeds_batch": (_I, [_P, _I32, _P, _P, _P, _P, _P]),
    "im_estimate_static": (_I, [_P, _P, _I64, _I32, _P, _I32, _P, _P]),
    "im_influence_mc": (_I, [_P, ctypes.POINTER(im_graph), _P, _I32, _I64, ctypes.c_uint64, _P, _P]),
    "im_server_create": (_I, [_P, ctypes.c_uint64, _I32, ctypes.POINTER(_P)]),
    "im_server_destroy": (_I, [_P]),
    "im_server_add_graph": (_I, [_P, ctypes.POINTER(im_graph), _P]),
    "im_server_submit": (_I, [_P, _I32, ctypes.POINTER(im_params), _P]),
    "im_server_step": (_I, [_P, _P, _P]),
    "im_server_footprint": (_I, [_P, _I32, ctypes.POINTER(im_params), _P]),
    "im_server_poll": (_I, [_P, ctypes.c_uint64, _P, _P, _P]),
    "im_server_cancel": (_I, [_P, ctypes.c_uint64]),
    "im_server_info": (_I, [_P, _P, _P, _P]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libim.so; raises if it has not been built (there is no fallback implementation)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"CUDA library {path} is missing: build it with paper_2105_04023_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib
