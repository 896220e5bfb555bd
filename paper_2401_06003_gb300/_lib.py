"""ctypes binding of libtrips.so, the C ABI declared in include/trips.h.

Argument marshalling only: every step of the splatting path runs in the
CUDA kernels behind these calls.  Loading fails loudly if the library has
not been built; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import build as _build

LIB_PATH = _build.LIB
HEADER = os.path.join(_build.INCLUDE, "trips.h")

(TP_OK, TP_ERR_INVALID_ARG, TP_ERR_CAPACITY, TP_ERR_NONFINITE, TP_ERR_TIMEOUT, TP_ERR_CUDA, TP_ERR_UNSUPPORTED,
 TP_ERR_BOUNDS) = range(8)
TP_FLAG_NONFINITE, TP_FLAG_CAPACITY, TP_FLAG_TIMEOUT, TP_FLAG_BOUNDS = 0x1, 0x2, 0x4, 0x8
TP_F32, TP_BF16 = 0, 1
TP_STORE_LISTS, TP_RECOMPUTE = 0, 1
TP_COARSE_LAYERS, TP_GRADS_ZEROED = 0x1, 0x2


class tp_camera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("znear", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class tp_config(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("K", ctypes.c_int32), ("desc_dim", ctypes.c_int32),
                ("eps", ctypes.c_float), ("desc_dtype", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("flags", ctypes.c_int32)]


class TripsError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed: {msg} (status {status})")
        self.status = status


_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "tp_pyramid_pixels": (_I64, [ctypes.POINTER(tp_camera), ctypes.c_int32, _P]),
    "tp_workspace_bytes": (_I64, [ctypes.POINTER(tp_config), ctypes.POINTER(tp_camera), _I64, _I64]),
    "tp_project": (ctypes.c_int, [ctypes.POINTER(tp_config), ctypes.POINTER(tp_camera), _I64, _P, _P, _P, _P, _I64,
                                  _P]),
    "tp_splat_forward": (ctypes.c_int, [ctypes.POINTER(tp_config), ctypes.POINTER(tp_camera), _I64, _P, _P, _P,
                                        _I64, _P]),
    "tp_blend": (ctypes.c_int, [ctypes.POINTER(tp_config), ctypes.POINTER(tp_camera), _I64, _P, _P, _P, _P, _P, _P,
                                _P, _P, _P, _I64, _P]),
    "tp_splat_backward": (ctypes.c_int, [ctypes.POINTER(tp_config), ctypes.POINTER(tp_camera), _I64, _P, _P, _P, _P,
                                         _P, _P, _P, _P, _P, _P, _P, _I64, _P]),
    "tp_batch_pixels": (_I64, [_P, ctypes.c_int32, ctypes.c_int32, _P]),
    "tp_batch_workspace_bytes": (_I64, [ctypes.POINTER(tp_config), _P, _P, ctypes.c_int32, _I64, _I64]),
    "tp_batch_project": (ctypes.c_int, [ctypes.POINTER(tp_config), _P, _P, ctypes.c_int32, _I64, _P, _P, _P, _P,
                                        _I64, _P]),
    "tp_batch_splat_forward": (ctypes.c_int, [ctypes.POINTER(tp_config), _P, _P, ctypes.c_int32, _I64, _P, _P, _P,
                                              _I64, _P]),
    "tp_batch_blend": (ctypes.c_int, [ctypes.POINTER(tp_config), _P, _P, ctypes.c_int32, _I64, _P, _P, _P, _P, _P,
                                      _P, _P, _P, _P, _I64, _P]),
    "tp_batch_splat_backward": (ctypes.c_int, [ctypes.POINTER(tp_config), _P, _P, ctypes.c_int32, _I64, _P, _P, _P,
                                               _P, _P, _P, _P, _P, _P, _P, _P, _I64, _P]),
    "tp_batch_splat_backward_cameras": (ctypes.c_int, [ctypes.POINTER(tp_config), _P, _P, ctypes.c_int32, _I64,
                                                       _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I64, _P]),
    "tp_zero_gradients": (ctypes.c_int, [ctypes.POINTER(tp_config), _I64, _P, _P, _P, _P, _P]),
    "tp_camera_backward": (ctypes.c_int, [ctypes.POINTER(tp_camera), _I64, _P, _P, _P, _P, _P, _P]),
    "tp_init_sizes_workspace_bytes": (_I64, [_I64]),
    "tp_init_point_sizes": (ctypes.c_int, [_I64, _P, _P, _P, _I64, _P]),
    "tp_merge": (ctypes.c_int, [ctypes.POINTER(tp_camera), ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "tp_merge_backward": (ctypes.c_int, [ctypes.POINTER(tp_camera), ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "tp_render_forward_static": (ctypes.c_int, [ctypes.POINTER(tp_config), ctypes.POINTER(tp_camera), _I64, _P, _P,
                                                _P, _P, _P, _P, _P, _P]),
    "tp_spatial_order_workspace_bytes": (_I64, [_I64]),
    "tp_spatial_order": (ctypes.c_int, [_I64, _P, _P, _P, _I64, _P]),
    "tp_permute_rows": (ctypes.c_int, [_I64, ctypes.c_int32, _P, _P, _P, _P]),
    "tp_get_status": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int32)]),
    "tp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tp_version": (ctypes.c_int32, []),
}


def header_functions() -> list[str]:
    """Names of the functions include/trips.h declares."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tp_[a-z_0-9]+)\s*\(", text)))


def load(path: str | None = None):
    """Load libtrips.so (built by ``paper_2401_06003_gb300.build``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libtrips.so is not built ({p}); run paper_2401_06003_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def check(fn: str, status: int):
    if status != TP_OK:
        msg = load().tp_status_string(status).decode()
        raise TripsError(fn, status, msg)


def make_camera(cam) -> tp_camera:
    """tp_camera from a scenes.Camera (or anything with its attributes)."""
    c = tp_camera()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = [float(v) for v in list(getattr(cam.R, "reshape")(9))]
    t = [float(v) for v in list(getattr(cam.t, "reshape")(3))]
    c.R = (ctypes.c_float * 9)(*R)
    c.t = (ctypes.c_float * 3)(*t)
    c.znear = float(cam.znear)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def make_config(n_layers: int, K: int, D: int, eps: float = 0.25, desc_dtype: int = TP_F32,
                mode: int = TP_RECOMPUTE, tile_w: int = 0, tile_h: int = 0, flags: int = 0) -> tp_config:
    return tp_config(int(n_layers), int(K), int(D), float(eps), int(desc_dtype), int(mode), int(tile_w), int(tile_h),
                     int(flags))
