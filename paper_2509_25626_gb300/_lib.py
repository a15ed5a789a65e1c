"""ctypes view of the C ABI in include/gs.h.

Loads the in-tree libgs.so.  There is no fallback: if the library is missing
or fails to load, every entry point raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs.so")

GS_OK = 0
GS_ERR_INVALID_ARG = -1
GS_ERR_CAPACITY = -2
GS_ERR_CUDA = -3
GS_ERR_TIMEOUT = -4
GS_ERR_TOO_LARGE = -5
SORT_STATIC_MAX_GAUSSIANS = 1 << 19
SORT_STATIC_MAX_INSTANCES = 1 << 21

c_float, c_int32, c_int64, c_void_p, c_size_t = (ctypes.c_float, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                                 ctypes.c_size_t)


class GsCamera(ctypes.Structure):
    _fields_ = [("viewmat", c_float * 16), ("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("width", c_int32), ("height", c_int32), ("tan_fovx", c_float), ("tan_fovy", c_float)]


class GsScene(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p), ("opacity_logits", c_void_p),
                ("sh", c_void_p), ("n", c_int64), ("sh_degree", c_int32), ("reserved", c_int32)]


# numpy view of one gs_splat record (64 bytes)
SPLAT_DTYPE = np.dtype([
    ("x", "<f4"), ("y", "<f4"), ("w00", "<f4"), ("w01", "<f4"), ("w11", "<f4"), ("log2_opacity", "<f4"),
    ("r", "<f4"), ("g", "<f4"), ("b", "<f4"), ("cull_hx", "<f4"), ("cull_hy", "<f4"), ("radius", "<i4"),
    ("depth", "<f4"), ("tiles_touched", "<u4"), ("rect_lo", "<u4"), ("rect_hi", "<u4"),
])
assert SPLAT_DTYPE.itemsize == 64


class GsSceneGrads(ctypes.Structure):
    _fields_ = [("dmeans", c_void_p), ("dlog_scales", c_void_p), ("dquats", c_void_p),
                ("dopacity_logits", c_void_p), ("dsh", c_void_p)]


class GsBalanceParams(ctypes.Structure):
    _fields_ = [("heavy_len", c_int32), ("max_heavy_tiles", c_int32), ("budget", c_int32),
                ("max_split_tiles", c_int32), ("max_chunks", c_int32), ("chunk", c_int32)]


class GsError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} (code {code})")
        self.code = code


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_2509_25626_gb300.build` "
                               "(or __graft_entry__.build()) on a machine with nvcc")
        L = ctypes.CDLL(LIB_PATH)
        P = c_void_p
        L.gs_preprocess.argtypes = [ctypes.POINTER(GsScene), ctypes.POINTER(GsCamera), P, P]
        L.gs_sort_workspace_bytes.argtypes = [c_int64, c_int64, c_int32]
        L.gs_sort_workspace_bytes.restype = c_size_t
        L.gs_sort.argtypes = [P, c_int64, ctypes.POINTER(GsCamera), P, P, c_int64, P, P, c_size_t,
                              ctypes.POINTER(c_int64), P]
        L.gs_sort_status.argtypes = [P, ctypes.POINTER(c_int64), P]
        L.gs_render.argtypes = [P, P, P, ctypes.POINTER(GsCamera), ctypes.POINTER(c_float), P, P, P, P]
        L.gs_sort_static.argtypes = [P, c_int64, ctypes.POINTER(GsCamera), P, P, c_int64, P,
                                     ctypes.POINTER(c_int64), P]
        L.gs_sort_static.restype = ctypes.c_int
        L.gs_render_batch.argtypes = [P, P, ctypes.c_int32, P]
        L.gs_render_batch.restype = ctypes.c_int
        L.gs_render_contrib.argtypes = [P, P, P, ctypes.POINTER(GsCamera), ctypes.POINTER(c_float), P, P, P, P]
        L.gs_render_contrib.restype = ctypes.c_int
        L.gs_render_workload.argtypes = [P, P, P, ctypes.POINTER(GsCamera), ctypes.POINTER(c_float), P, P, P, P, P, P]
        L.gs_render_ex.argtypes = [P, P, P, ctypes.POINTER(GsCamera), ctypes.POINTER(c_float)] + [P] * 7
        L.gs_splat_buffer_bytes.argtypes = [ctypes.c_int64]
        L.gs_frame.argtypes = [ctypes.POINTER(GsScene), ctypes.POINTER(GsCamera), P, P, P, ctypes.c_int64, P, P,
                               c_size_t, ctypes.POINTER(c_float), P, P, P, P]
        L.gs_frame.restype = ctypes.c_int
        L.gs_splat_buffer_bytes.restype = c_size_t
        L.gs_backward_workspace_bytes.argtypes = [c_int64]
        L.gs_backward_workspace_bytes.restype = c_size_t
        L.gs_render_backward.argtypes = [ctypes.POINTER(GsScene), ctypes.POINTER(GsCamera), P, P, P,
                                         ctypes.POINTER(c_float), P, P, P, P, c_size_t,
                                         ctypes.POINTER(GsSceneGrads), P]
        L.gs_render_backward.restype = ctypes.c_int
        L.gs_render_backward_splats.argtypes = [ctypes.POINTER(GsCamera), P, c_int64, P, P, ctypes.POINTER(c_float),
                                                P, P, P, P, P]
        L.gs_render_backward_splats.restype = ctypes.c_int
        L.gs_preprocess_backward.argtypes = [ctypes.POINTER(GsScene), ctypes.POINTER(GsCamera), P, P,
                                             ctypes.POINTER(GsSceneGrads), P]
        L.gs_preprocess_backward.restype = ctypes.c_int
        L.gs_render_balance_workspace_bytes.argtypes = [ctypes.POINTER(GsBalanceParams)]
        L.gs_render_balance_workspace_bytes.restype = c_size_t
        L.gs_render_batch_balanced.argtypes = [P, P, ctypes.POINTER(GsBalanceParams), P, c_size_t, ctypes.c_int32, P]
        L.gs_render_batch_balanced.restype = ctypes.c_int
        L.gs_camera_block_bytes.argtypes = []
        L.gs_camera_block_bytes.restype = c_size_t
        L.gs_camera_block.argtypes = [ctypes.POINTER(GsCamera), P]
        L.gs_camera_block.restype = ctypes.c_int
        L.gs_preprocess_camblock.argtypes = [ctypes.POINTER(GsScene), P, P, P]
        L.gs_preprocess_camblock.restype = ctypes.c_int
        L.gs_check_wait_timeout.argtypes = [P, c_size_t, ctypes.c_uint64, P]
        L.gs_check_wait_timeout.restype = ctypes.c_int
        L.gs_strerror.argtypes = [ctypes.c_int]
        L.gs_strerror.restype = ctypes.c_char_p
        L.gs_last_cuda_error.restype = ctypes.c_char_p
        for name in ("gs_preprocess", "gs_sort", "gs_sort_status", "gs_render", "gs_render_workload", "gs_render_ex",
                     "gs_version", "gs_built_arch"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().gs_strerror(int(code)).decode()


def check(code: int, what: str) -> int:
    if code != GS_OK:
        raise GsError(code, what)
    return code


def exported_symbols():
    """Names of the gs_* functions the header declares."""
    return ["gs_splat_buffer_bytes", "gs_frame", "gs_preprocess", "gs_camera_block_bytes", "gs_camera_block",
            "gs_preprocess_camblock", "gs_sort_workspace_bytes", "gs_sort", "gs_sort_status", "gs_render",
            "gs_render_workload", "gs_render_ex", "gs_render_contrib", "gs_sort_static", "gs_backward_workspace_bytes",
            "gs_render_backward", "gs_render_backward_splats", "gs_preprocess_backward",
            "gs_render_batch", "gs_render_balance_workspace_bytes", "gs_render_batch_balanced", "gs_check_wait_timeout",
            "gs_strerror", "gs_last_cuda_error", "gs_version", "gs_built_arch"]
