"""ctypes declarations of the C ABI in include/cygrid_gb300.h (same names).

Argument marshalling only: every step of the gridding runs in the CUDA
library.  There is no fallback: if the library has not been built, importing
this module raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libcygrid_gb300.so")

CG_OK, CG_EINVAL, CG_ENOMEM, CG_ECUDA, CG_EDEVICE, CG_ETIMEOUT, CG_ESTATE = range(7)
CG_F32, CG_BF16 = 0, 1
CG_GAUSS1D, CG_GAUSS2D, CG_TSINC = 0, 1, 2
CG_PATH_AUTO, CG_PATH_FP32, CG_PATH_TC, CG_PATH_TC_FAST = 0, 1, 2, 3

STATUS_NAMES = {0: "CG_OK", 1: "CG_EINVAL", 2: "CG_ENOMEM", 3: "CG_ECUDA", 4: "CG_EDEVICE",
                5: "CG_ETIMEOUT", 6: "CG_ESTATE"}


class CgInfo(ctypes.Structure):
    _fields_ = [("n_targets", ctypes.c_int64), ("n_channels", ctypes.c_int32),
                ("nside", ctypes.c_int32), ("n_tiles", ctypes.c_int64),
                ("tile_size", ctypes.c_int32), ("path", ctypes.c_int32),
                ("n_ranges", ctypes.c_int64), ("n_samples_total", ctypes.c_int64),
                ("n_pairs", ctypes.c_int64), ("n_launches", ctypes.c_int64),
                ("n_candidates", ctypes.c_int64)]

CG_N_STAGES = 5
STAGE_NAMES = ("keys", "sort", "index", "grid", "finalize")


class CgJob(ctypes.Structure):
    """cg_job of include/cygrid_gb300.h."""
    _fields_ = [("grid", ctypes.c_void_p), ("lon_deg", ctypes.c_void_p),
                ("lat_deg", ctypes.c_void_p), ("data", ctypes.c_void_p),
                ("data_dtype", ctypes.c_int32), ("weights", ctypes.c_void_p),
                ("n_samples", ctypes.c_int64), ("out", ctypes.c_void_p),
                ("layout_channel_major", ctypes.c_int32), ("out_weights", ctypes.c_void_p)]


class CygridError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double

# name -> argtypes; every function returns cg_status (int) except cg_last_error
SIGNATURES = {
    "cg_grid_create": [ctypes.POINTER(_vp), _vp, _vp, _i64, _i32, _vp],
    "cg_set_kernel": [_vp, _i32, ctypes.POINTER(_dbl), _i32, _dbl, _i32, _dbl],
    "cg_grid_add": [_vp, _vp, _vp, _vp, _i32, _vp, _i64],
    "cg_grid_finalize": [_vp, _vp, _i32, _vp],
    "cg_grid_oneshot": [_vp, _vp, _vp, _vp, _i32, _vp, _i64, _vp, _i32, _vp],
    "cg_grid_oneshot_host": [_vp, _vp, _vp, _vp, _i32, _vp, _i64, _vp, _i32, _vp],
    "cg_grid_oneshot_pcw": [_vp, _vp, _vp, _vp, _i32, _vp, _i64, _vp, _i32, _vp],
    "cg_interp": [_vp, _vp, _vp, _vp, _i64],
    "cg_grid_reset": [_vp],
    "cg_grid_destroy": [_vp],
    "cg_set_stream": [_vp, _vp],
    "cg_set_path": [_vp, _i32],
    "cg_sync": [_vp],
    "cg_get_info": [_vp, ctypes.POINTER(CgInfo)],
    "cg_ang2pix_ring": [_i32, _vp, _vp, _i64, _vp, _vp],
    "cg_unit_vectors": [_vp, _vp, _i64, _vp, _vp],
    "cg_set_f32_shape": [_vp, _i32],
    "cg_degrid": [_vp, _vp, _vp, _vp, _i64],
    "cg_grid_dsigma": [_vp, _vp, _i32, _vp, _vp, _vp],
    "cg_grid_export_index": [_vp, _vp, _vp, _vp, _i64],
    "cg_set_timing": [_vp, _i32],
    "cg_read_timing": [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_i64)],
    "cg_debug_hold": [_vp, _i32, _i64],
    "cg_sort_samples_noalloc": [_i32, _vp, _vp, _i64, _vp, _vp, _vp],
    "cg_batch_create": [ctypes.POINTER(_vp), ctypes.POINTER(CgJob), _i32, _i32],
    "cg_batch_autotune": [_vp, _i32, _i32],
    "cg_batch_capture": [_vp, _vp],
    "cg_batch_run": [_vp, _vp],
    "cg_batch_get_choice": [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                            ctypes.POINTER(_dbl), ctypes.POINTER(_i32)],
    "cg_batch_info": [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32)],
    "cg_batch_destroy": [_vp],
    "cg_batch_set_fused": [_vp, _i32],
    "cg_md_residual": [_vp, _vp, _vp, _i64, _vp],
    "cg_md_update": [_vp, _vp, _vp, ctypes.c_float, _i64],
    "cg_batch_sync": [_vp],
    "cg_batch_debug_hold": [_vp, _i32, _i64],
}

CG_NOALLOC_MAX_SAMPLES = 262144

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libcygrid_gb300.so is not built (%s); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.cg_last_error.argtypes = []
    lib.cg_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(status: int):
    if status != CG_OK:
        msg = load().cg_last_error()
        raise CygridError(status, msg.decode() if msg else "")
    return status


def _call(name):
    def f(*args):
        return check(getattr(load(), name)(*args))
    f.__name__ = name
    return f


cg_grid_create = _call("cg_grid_create")
cg_set_kernel = _call("cg_set_kernel")
cg_grid_add = _call("cg_grid_add")
cg_grid_finalize = _call("cg_grid_finalize")
cg_grid_oneshot = _call("cg_grid_oneshot")
cg_grid_oneshot_host = _call("cg_grid_oneshot_host")
cg_grid_oneshot_pcw = _call("cg_grid_oneshot_pcw")
cg_interp = _call("cg_interp")
cg_grid_reset = _call("cg_grid_reset")
cg_grid_destroy = _call("cg_grid_destroy")
cg_set_stream = _call("cg_set_stream")
cg_set_path = _call("cg_set_path")
cg_sync = _call("cg_sync")
cg_get_info = _call("cg_get_info")
cg_ang2pix_ring = _call("cg_ang2pix_ring")
cg_unit_vectors = _call("cg_unit_vectors")
cg_set_f32_shape = _call("cg_set_f32_shape")
cg_degrid = _call("cg_degrid")
cg_grid_dsigma = _call("cg_grid_dsigma")
cg_grid_export_index = _call("cg_grid_export_index")
cg_set_timing = _call("cg_set_timing")
cg_read_timing = _call("cg_read_timing")
cg_sort_samples_noalloc = _call("cg_sort_samples_noalloc")
cg_debug_hold = _call("cg_debug_hold")
cg_batch_create = _call("cg_batch_create")
cg_batch_autotune = _call("cg_batch_autotune")
cg_batch_capture = _call("cg_batch_capture")
cg_batch_run = _call("cg_batch_run")
cg_batch_get_choice = _call("cg_batch_get_choice")
cg_batch_info = _call("cg_batch_info")
cg_batch_destroy = _call("cg_batch_destroy")
cg_batch_set_fused = _call("cg_batch_set_fused")
cg_md_residual = _call("cg_md_residual")
cg_md_update = _call("cg_md_update")
cg_batch_sync = _call("cg_batch_sync")
cg_batch_debug_hold = _call("cg_batch_debug_hold")


def cg_last_error() -> str:
    return load().cg_last_error().decode()
