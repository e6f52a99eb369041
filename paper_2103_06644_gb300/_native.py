"""ctypes binding of libsurffit.so: argument marshalling only.

Every computation runs in the CUDA library.  Loading fails loudly when the
library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SF_OK = 0
STATUS = {0: "SF_OK", 1: "SF_ERR_INVALID_ARG", 2: "SF_ERR_UNSUPPORTED", 3: "SF_ERR_ALLOC", 4: "SF_ERR_CUDA",
          5: "SF_ERR_TIMEOUT"}


class SurfFitError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, str(status)), msg))
        self.status = status


class Intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double)]


class BatchFrame(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("window", ctypes.c_int), ("K", Intrinsics),
                ("depth", ctypes.c_void_p), ("normals", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("curvature", ctypes.c_void_p), ("hseg", ctypes.c_int), ("vband", ctypes.c_int)]


_lib = None

# name -> (restype, argtypes)
_VP = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
class QuadParams(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("max_level", ctypes.c_int), ("tau", ctypes.c_float),
                ("min_valid_permille", ctypes.c_int)]


# sf_quad_node as a numpy record (56 bytes)
QUAD_NODE_DTYPE = [("frame", "<i4"), ("x0", "<i4"), ("y0", "<i4"), ("w", "<i4"), ("h", "<i4"), ("level", "<i4"),
                   ("status", "<i4"), ("count", "<i4"), ("normal", "<f4", (3,)), ("offset", "<f4"),
                   ("curvature", "<f4"), ("rms", "<f4")]

SIGNATURES = {
    "sf_create": (_I, [ctypes.POINTER(Intrinsics), _I, _I, _I, ctypes.POINTER(_VP)]),
    "sf_set_params": (_I, [_VP, _I, _I, _F, _I, _I]),
    "sf_fit": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "sf_fit_ex": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sf_fit_host": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sf_destroy": (_I, [_VP]),
    "sf_set_precision": (_I, [_VP, _I, _F]),
    "sf_precision_stats": (_I, [_VP, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)]),
    "sf_set_constraint": (_I, [_VP, _I]),
    "sf_set_disparity_model": (_I, [_VP, ctypes.c_double, ctypes.c_double]),
    "sf_set_tiles": (_I, [_VP, _I, _I]),
    "sf_set_delta_table": (_I, [_VP, _VP, _VP]),
    "sf_batch_create": (_I, [ctypes.POINTER(BatchFrame), _I, _I, _I, _F, _I, _I, _I, ctypes.POINTER(_VP)]),
    "sf_batch_run": (_I, [_VP, _VP]),
    "sf_batch_info": (_I, [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_I)]),
    "sf_batch_destroy": (_I, [_VP]),
    "sf_fit_backward": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sf_fit_backward_ex": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP, ctypes.c_uint, _VP]),
    "sf_backward_reuses": (_I, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
    "sf_last_error": (ctypes.c_char_p, []),
    "sf_channel_counts": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "sf_version": (ctypes.c_char_p, []),
    "sf_eval_acos": (_I, [_VP, _VP, _I, _VP]),
    "sf_batch_check": (_I, [_VP]),
    "sf_debug_fail_allocs": (_I, [ctypes.c_longlong]),
    "sf_debug_live_allocs": (_I, [ctypes.POINTER(ctypes.c_longlong)]),
    "sf_graph_replays": (_I, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    "sf_batch_set_wait_limit": (_I, [_VP, ctypes.c_uint]),
    "sf_profile_enable": (_I, [_VP, _I]),
    "sf_profile_read": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I)]),
    "sf_fit_static": (_I, [ctypes.POINTER(Intrinsics), _I, _I, _I, _I, _I, _F, _I, _I, _VP, _VP, _VP, _VP, _VP]),
    "sf_quadtree": (_I, [_VP, _I, _VP, ctypes.POINTER(QuadParams), _VP, _I, _VP, _VP]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libsurffit.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libsurffit.so is not built (%s); run paper_2103_06644_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != SF_OK:
        raise SurfFitError(status, lib().sf_last_error().decode())
