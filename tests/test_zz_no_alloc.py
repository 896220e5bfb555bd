"""tp_render_forward_static: the forward render for callers that may not
allocate device memory at run time (a plug-in whose host application owns
all CUDA allocations, a frame loop that must not call cudaMalloc once it
runs).  Its workspace is an array the library reserves on each device, so
the test checks that it renders what tp_project + tp_splat_forward +
tp_blend render with a caller workspace, on two calls in a row that share
that array (the second call smaller than the first, so leftovers of the
first would show), and that a frame too large for the array is refused.

The file name sorts last so pytest runs it after the other tests; it also
passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_helpers import PYR_RTOL, assert_close_scaled, device, to_dev
from paper_2401_06003_gb300 import Renderer, _lib, scenes

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _static_render(r, pos, sw, op, desc):
    """One call of the allocation-free entry point with the renderer's settings."""
    lib = _lib.load()
    n = pos.shape[0]
    records = torch.full((n, 4), float("nan"), device=device())
    pyramid = torch.full((r.P, r.D), float("nan"), device=device())
    flags = torch.full((1,), 0x7FFFFFFF, dtype=torch.int32, device=device())
    stream = ctypes.c_void_p(torch.cuda.current_stream(device()).cuda_stream)
    st = lib.tp_render_forward_static(ctypes.byref(r.cfg), ctypes.byref(r.cam), n, _ptr(pos), _ptr(sw), _ptr(op),
                                      _ptr(desc), _ptr(records), _ptr(pyramid), _ptr(flags), stream)
    _lib.check("tp_render_forward_static", st)
    torch.cuda.synchronize()
    return records, pyramid, int(flags.item())


def _case(n, seed, width, height, n_layers, K, D, desc_dtype):
    sc = scenes.scene_uniform_cube(n=n, seed=seed, res=64)
    cam = scenes.camera_at((0.4, 0.3, -2.6), (0.0, 0.0, 0.0), width, height)
    rng = np.random.default_rng(seed + 100)
    desc = to_dev(rng.uniform(-1, 1, (n, D)), dtype=desc_dtype)
    r = Renderer(cam, n_layers, K=K, D=D, desc_dtype=desc_dtype, mode="store", device=device())
    return r, to_dev(sc.pos), to_dev(sc.size_w), to_dev(sc.opacity), desc


def test_static_workspace_matches_caller_workspace_twice():
    cases = [_case(20000, 11, 256, 192, 5, 16, 4, torch.float32),
             _case(3000, 12, 120, 72, 4, 8, 8, torch.bfloat16)]
    for call, (r, pos, sw, op, desc) in enumerate(cases):
        records, pyramid, flags = _static_render(r, pos, sw, op, desc)
        ref = r.render(pos, sw, op, desc)
        assert r.status(ref.workspace) == 0
        assert flags == 0, f"call {call}: device flags {flags:#x}"
        assert torch.equal(records, ref.records), f"call {call}: records"
        assert_close_scaled(pyramid.cpu().numpy(), ref.pyramid.cpu().numpy(), PYR_RTOL, name=f"call {call} pyramid")


def test_static_workspace_refuses_oversized_frame():
    lib = _lib.load()
    cam = _lib.make_camera(scenes.camera_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 1920, 1080))
    cfg = _lib.make_config(8, 16, 4)
    n = 1_000_000
    assert lib.tp_workspace_bytes(ctypes.byref(cfg), ctypes.byref(cam), n, 0) > 64 << 20
    st = lib.tp_render_forward_static(ctypes.byref(cfg), ctypes.byref(cam), n, None, None, None, None, None, None,
                                      None, None)
    assert st == _lib.TP_ERR_CAPACITY
