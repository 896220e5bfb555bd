"""The C-ABI library builds, loads and exports every declared symbol; host-only logic.

Nothing here launches a kernel: the calls exercised are the pure host
functions (layout, workspace size, argument checks that fail before any
CUDA call) and the status strings.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2401_06003_gb300 import _lib, scenes
from paper_2401_06003_gb300.build import build


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    names = _lib.header_functions()
    assert {"tp_project", "tp_splat_forward", "tp_blend", "tp_splat_backward"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name
    assert set(_lib._SIGS) == set(names), "binding and header disagree"
    assert lib.tp_version() >= 100


def test_checking_build_exports_every_declared_symbol():
    """libtrips_debug.so (TP_DEBUG index checks) is the same ABI."""
    dbg = _lib.load(build(debug=True))
    for name in _lib.header_functions():
        assert hasattr(dbg, name), name
    assert dbg.tp_status_string(_lib.TP_ERR_BOUNDS).decode().startswith("out-of-range")


def test_zero_gradients_host_checks(lib):
    cfg = _lib.make_config(4, 16, 4)
    assert lib.tp_zero_gradients(ctypes.byref(cfg), 0, None, None, None, None, None) == _lib.TP_OK
    assert lib.tp_zero_gradients(ctypes.byref(cfg), 10, None, None, None, None, None) == _lib.TP_ERR_INVALID_ARG
    assert lib.tp_zero_gradients(ctypes.byref(cfg), -1, None, None, None, None, None) == _lib.TP_ERR_INVALID_ARG
    bad = _lib.make_config(4, 16, 4, flags=0x4)
    assert lib.tp_zero_gradients(ctypes.byref(bad), 0, None, None, None, None, None) == _lib.TP_ERR_INVALID_ARG


def test_struct_layout_matches_header():
    assert ctypes.sizeof(_lib.tp_camera) == 17 * 4 + 2 * 4
    assert ctypes.sizeof(_lib.tp_config) == 9 * 4


def test_coarse_layer_flag(lib):
    """Coarse-layer inclusion adds K slots (8-byte key, 4-byte opacity) per
    pixel of layers >= 1 to the workspace; unknown flag bits are refused; a
    stored-lists backward with inclusion is refused before any CUDA call."""
    sc = scenes.make_config("cube20k_256", n=10)
    cam = _lib.make_camera(sc.camera)
    offs, _, _ = oracle.pyramid_layout(sc.camera.width, sc.camera.height, 4)
    coarse_pix = int(offs[-1] - offs[1])
    for K in (4, 16, 32):
        plain = _lib.make_config(4, K, 4)
        coarse = _lib.make_config(4, K, 4, flags=_lib.TP_COARSE_LAYERS)
        a = lib.tp_workspace_bytes(ctypes.byref(plain), ctypes.byref(cam), 1000, 0)
        b = lib.tp_workspace_bytes(ctypes.byref(coarse), ctypes.byref(cam), 1000, 0)
        assert 0 <= (b - a) - 12 * K * coarse_pix < 512, (K, a, b)
    bad = _lib.make_config(4, 16, 4, flags=0x4)
    assert lib.tp_workspace_bytes(ctypes.byref(bad), ctypes.byref(cam), 10, 0) == -1
    coarse = _lib.make_config(4, 16, 4, mode=_lib.TP_STORE_LISTS, flags=_lib.TP_COARSE_LAYERS)
    need = lib.tp_workspace_bytes(ctypes.byref(coarse), ctypes.byref(cam), 10, 0)
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: the call fails in its host checks
    st = lib.tp_splat_backward(ctypes.byref(coarse), ctypes.byref(cam), 10, fake, fake, fake, fake, fake, fake,
                               fake, fake, fake, fake, fake, need, None)
    assert st == _lib.TP_ERR_UNSUPPORTED


@pytest.mark.parametrize("W,H,L", [(256, 256, 4), (1920, 1080, 8), (257, 131, 3), (3840, 2160, 10), (1, 1, 1)])
def test_pyramid_pixels_matches_oracle_layout(lib, W, H, L):
    cam = scenes.Camera(W, W, W / 2, H / 2, np.eye(3), np.zeros(3), W, H)
    offs = (ctypes.c_int64 * (L + 1))()
    P = lib.tp_pyramid_pixels(ctypes.byref(_lib.make_camera(cam)), L, offs)
    ref, _, _ = oracle.pyramid_layout(W, H, L)
    assert P == ref[-1]
    assert list(offs) == ref.tolist()


def test_workspace_bytes_and_checks(lib):
    cam = _lib.make_camera(scenes.make_config("cube20k_256", n=10).camera)
    cfg = _lib.make_config(4, 16, 4)
    b8 = lib.tp_workspace_bytes(ctypes.byref(cfg), ctypes.byref(cam), 1000, 0)
    b1 = lib.tp_workspace_bytes(ctypes.byref(cfg), ctypes.byref(cam), 1000, 1000)
    assert b8 > b1 > 0 and (b8 - b1) >= 7000 * 20 - 512
    bad = _lib.make_config(4, 12, 4)  # K = 12 is not instantiated
    assert lib.tp_workspace_bytes(ctypes.byref(bad), ctypes.byref(cam), 10, 0) == -1
    bad = _lib.make_config(0, 16, 4)
    assert lib.tp_workspace_bytes(ctypes.byref(bad), ctypes.byref(cam), 10, 0) == -1
    # argument errors come back before any CUDA call
    st = lib.tp_project(ctypes.byref(cfg), ctypes.byref(cam), 10, None, None, None, None, 0, None)
    assert st == _lib.TP_ERR_INVALID_ARG
    st = lib.tp_project(ctypes.byref(_lib.make_config(4, 12, 4)), ctypes.byref(cam), 10, None, None, None,
                        None, 0, None)
    assert st == _lib.TP_ERR_UNSUPPORTED
    cam.znear = 0.0
    st = lib.tp_splat_forward(ctypes.byref(cfg), ctypes.byref(cam), 10, None, None, None, 0, None)
    assert st == _lib.TP_ERR_INVALID_ARG
    assert lib.tp_status_string(_lib.TP_ERR_CAPACITY).decode().startswith("workspace")


def test_size_limits_are_refused_on_the_host(lib):
    """Documented maxima: n < 2^27 points, 16 layers, D <= 64, width and height <= 32768."""
    cam = _lib.make_camera(scenes.make_config("cube20k_256", n=10).camera)
    cfg = _lib.make_config(4, 16, 4)
    assert lib.tp_workspace_bytes(ctypes.byref(cfg), ctypes.byref(cam), (1 << 27) - 1, 1) > 0
    assert lib.tp_workspace_bytes(ctypes.byref(cfg), ctypes.byref(cam), 1 << 27, 1) == -1
    assert lib.tp_workspace_bytes(ctypes.byref(_lib.make_config(16, 16, 4)), ctypes.byref(cam), 10, 0) > 0
    assert lib.tp_workspace_bytes(ctypes.byref(_lib.make_config(17, 16, 4)), ctypes.byref(cam), 10, 0) == -1
    assert lib.tp_workspace_bytes(ctypes.byref(_lib.make_config(4, 16, 64)), ctypes.byref(cam), 10, 0) > 0
    assert lib.tp_workspace_bytes(ctypes.byref(_lib.make_config(4, 16, 65)), ctypes.byref(cam), 10, 0) == -1
    wide = _lib.make_camera(scenes.camera_at((0, 0, -3), (0, 0, 0), 32768, 2))
    assert lib.tp_workspace_bytes(ctypes.byref(cfg), ctypes.byref(wide), 10, 0) > 0
    wide.width = 32769
    assert lib.tp_workspace_bytes(ctypes.byref(cfg), ctypes.byref(wide), 10, 0) == -1


def test_batch_entry_offsets_stay_32_bit(lib):
    """A batch may hold at most 8 (point, tile) entries per point and view below 2^32:
    n x views < 2^29 (the tile offsets are 32-bit)."""
    cams = (_lib.tp_camera * 16)(*[_lib.make_camera(scenes.make_config("cube20k_256", n=10).camera)] * 16)
    cfg = _lib.make_config(4, 16, 4)
    assert lib.tp_batch_workspace_bytes(ctypes.byref(cfg), cams, None, 16, (1 << 25) - 1, 1) > 0
    assert lib.tp_batch_workspace_bytes(ctypes.byref(cfg), cams, None, 16, 1 << 25, 1) == -1
    assert lib.tp_batch_workspace_bytes(ctypes.byref(cfg), cams, None, 8, (1 << 27) - 1, 1) == -1
    assert lib.tp_batch_workspace_bytes(ctypes.byref(cfg), cams, None, 2, (1 << 27) - 1, 1) > 0
