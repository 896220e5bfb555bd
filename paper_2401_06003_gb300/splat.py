"""Thin torch layer over the C ABI: device buffers, streams and autograd.

Every step of the splatting path (projection, binning, per-pixel top-K,
blending and the adjoint) runs inside libtrips.so; this module only
allocates tensors, passes their pointers and the current CUDA stream, and
wires the backward call into ``torch.autograd``.
"""
from __future__ import annotations

import ctypes
import dataclasses

import torch

from . import _lib

_DTYPES = {torch.float32: _lib.TP_F32, torch.bfloat16: _lib.TP_BF16}


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _need(t, dtype, shape, name, device):
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous() or t.device != device:
        raise ValueError(f"{name}: expected contiguous {dtype} {tuple(shape)} on {device}, "
                         f"got {t.dtype} {tuple(t.shape)} on {t.device}")


def _grad_buffers(n, D, dev, grads):
    """Point-gradient buffers of a backward call: (pointers for the C call,
    tensors returned to the caller).  By default the position and size
    gradients share packed [n, 4] rows (one 16-byte atomic per fragment); the
    caller gets [n, 3] and [n] views of them.  ``grads`` may hold caller
    buffers: (pos [n, 3], size_w [n], opacity, desc), or (pos [n, 4] packed,
    None, opacity, desc)."""
    if grads is None:
        g4 = torch.empty((n, 4), dtype=torch.float32, device=dev)
        grads = (g4, None, torch.empty((n,), dtype=torch.float32, device=dev),
                 torch.empty((n, D), dtype=torch.float32, device=dev))
    gp, gs, go, gd = grads
    if tuple(gp.shape) == (n, 4):
        return (gp, None, go, gd), (gp[:, :3], gp[:, 3], go, gd)
    return (gp, gs, go, gd), (gp, gs, go, gd)


def _backward_cfg(cfg, grads_zeroed):
    """The frame's config, with TP_GRADS_ZEROED when the caller cleared the gradients."""
    if not grads_zeroed:
        return ctypes.byref(cfg)
    c = _lib.tp_config.from_buffer_copy(cfg)
    c.flags |= _lib.TP_GRADS_ZEROED
    return ctypes.byref(c)


def _packed_pos_size(grad_pos, grad_size_w):
    """The packed [n, 4] base of (grad_pos, grad_size_w) views, or None."""
    n = grad_pos.shape[0]
    if tuple(grad_pos.shape) == (n, 4) and grad_pos.is_contiguous():
        return grad_pos
    if (grad_size_w is not None and grad_pos.stride() == (4, 1) and grad_size_w.stride() == (4,)
            and grad_size_w.data_ptr() == grad_pos.data_ptr() + 12):
        return torch.as_strided(grad_pos, (n, 4), (4, 1))
    return None


@dataclasses.dataclass
class Frame:
    """Outputs of one forward render and what the backward pass needs."""

    pyramid: torch.Tensor       # [P, D] float32
    records: torch.Tensor       # [n, 4] float32 (x, y, z, s)
    workspace: torch.Tensor     # uint8, holds the frame's tile lists
    kept: torch.Tensor | None = None      # [P, K] int32 view of uint32 ids
    n_kept: torch.Tensor | None = None    # [P] uint8
    t_final: torch.Tensor | None = None   # [P] float32
    n_frag: torch.Tensor | None = None    # [P] int32 view of uint32 counts


class Renderer:
    """A camera plus render settings; renders point clouds through libtrips.so.

    ``mode``: "recompute" keeps only the tile lists between the forward and
    the backward pass and rebuilds each pixel's sorted list in the backward
    kernel; "store" keeps the per-pixel kept lists from the forward pass.
    ``coarse``: coarse-layer inclusion (Sec. 3.6): each pixel's list also
    holds the fragments of the coarser pixels that contain it (backward
    passes in "recompute" mode only).
    """

    def __init__(self, camera, n_layers: int, K: int = 16, D: int = 4, eps: float = 0.25,
                 desc_dtype=torch.float32, mode: str = "recompute", tile=(16, 8), device=None,
                 coarse: bool = False):
        self.lib = _lib.load()
        self.camera = camera
        self.cam = _lib.make_camera(camera)
        if desc_dtype not in _DTYPES:
            raise ValueError(f"descriptor dtype {desc_dtype} not supported")
        self.desc_dtype = desc_dtype
        self.mode = {"store": _lib.TP_STORE_LISTS, "recompute": _lib.TP_RECOMPUTE}[mode]
        self.coarse = bool(coarse)
        self.cfg = _lib.make_config(n_layers, K, D, eps, _DTYPES[desc_dtype], self.mode, tile[0], tile[1],
                                    _lib.TP_COARSE_LAYERS if coarse else 0)
        self.n_layers, self.K, self.D = int(n_layers), int(K), int(D)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        offs = (ctypes.c_int64 * (n_layers + 1))()
        P = self.lib.tp_pyramid_pixels(ctypes.byref(self.cam), n_layers, offs)
        if P < 0:
            raise ValueError("invalid camera or layer count")
        self.P = int(P)
        self.layer_offsets = [int(v) for v in offs]

    # -- sizes ---------------------------------------------------------------
    def workspace_bytes(self, n: int, capacity: int = 0) -> int:
        b = self.lib.tp_workspace_bytes(ctypes.byref(self.cfg), ctypes.byref(self.cam), int(n), int(capacity))
        if b < 0:
            raise ValueError("invalid configuration for the workspace")
        return int(b)

    def new_workspace(self, n: int, capacity: int = 0) -> torch.Tensor:
        ws = torch.empty(self.workspace_bytes(n, capacity), dtype=torch.uint8, device=self.device)
        assert ws.data_ptr() % 256 == 0
        return ws

    def layer(self, pyramid: torch.Tensor, L: int) -> torch.Tensor:
        """View of layer L of a [P, D] pyramid as [H_L, W_L, D]."""
        s = 1 << L
        w = -(-self.cam.width // s)
        h = -(-self.cam.height // s)
        return pyramid[self.layer_offsets[L]:self.layer_offsets[L + 1]].view(h, w, -1)

    # -- the four C-ABI stages -----------------------------------------------
    def project(self, pos, size_w, ws, records=None):
        n = pos.shape[0]
        _need(pos, torch.float32, (n, 3), "pos", self.device)
        _need(size_w, torch.float32, (n,), "size_w", self.device)
        if records is None:
            records = torch.empty((n, 4), dtype=torch.float32, device=self.device)
        st = self.lib.tp_project(ctypes.byref(self.cfg), ctypes.byref(self.cam), n, _ptr(pos), _ptr(size_w),
                                 _ptr(records), _ptr(ws), ws.numel(), _stream(self.device))
        _lib.check("tp_project", st)
        return records

    def splat_forward(self, records, opacity, ws):
        n = records.shape[0]
        _need(opacity, torch.float32, (n,), "opacity", self.device)
        st = self.lib.tp_splat_forward(ctypes.byref(self.cfg), ctypes.byref(self.cam), n, _ptr(records),
                                       _ptr(opacity), _ptr(ws), ws.numel(), _stream(self.device))
        _lib.check("tp_splat_forward", st)

    def blend(self, records, opacity, desc, ws, store_lists=False, stats=False, pyramid=None):
        n = records.shape[0]
        _need(records, torch.float32, (n, 4), "records", self.device)
        _need(opacity, torch.float32, (n,), "opacity", self.device)
        _need(desc, self.desc_dtype, (n, self.D), "desc", self.device)
        dev = self.device
        if pyramid is None:
            pyramid = torch.empty((self.P, self.D), dtype=torch.float32, device=dev)
        kept = n_kept = t_final = n_frag = None
        if store_lists or stats:
            kept = torch.empty((self.P, self.K), dtype=torch.int32, device=dev)
            n_kept = torch.empty((self.P,), dtype=torch.uint8, device=dev)
        if stats:
            t_final = torch.empty((self.P,), dtype=torch.float32, device=dev)
            n_frag = torch.empty((self.P,), dtype=torch.int32, device=dev)
        st = self.lib.tp_blend(ctypes.byref(self.cfg), ctypes.byref(self.cam), n, _ptr(records), _ptr(opacity),
                               _ptr(desc), _ptr(pyramid), _ptr(kept), _ptr(n_kept), _ptr(t_final), _ptr(n_frag),
                               _ptr(ws), ws.numel(), _stream(dev))
        _lib.check("tp_blend", st)
        return pyramid, kept, n_kept, t_final, n_frag

    def splat_backward(self, records, opacity, desc, grad_pyramid, ws, kept=None, n_kept=None, grads=None,
                       grads_zeroed=False):
        """Point gradients of sum(grad_pyramid * pyramid).  ``grads_zeroed``: the
        caller's ``grads`` buffers are already zero (cleared, e.g., on another
        stream during the forward kernels), so the call only adds to them."""
        n = records.shape[0]
        dev = self.device
        _need(grad_pyramid, torch.float32, (self.P, self.D), "grad_pyramid", dev)
        if grads_zeroed and grads is None:
            raise ValueError("grads_zeroed needs the caller's gradient buffers")
        (gp, gs, go, gd), out = _grad_buffers(n, self.D, dev, grads)
        st = self.lib.tp_splat_backward(_backward_cfg(self.cfg, grads_zeroed), ctypes.byref(self.cam), n,
                                        _ptr(records), _ptr(opacity), _ptr(desc), _ptr(kept), _ptr(n_kept), _ptr(grad_pyramid),
                                        _ptr(gp), _ptr(gs), _ptr(go), _ptr(gd), _ptr(ws), ws.numel(), _stream(dev))
        _lib.check("tp_splat_backward", st)
        return out

    def zero_gradients(self, grads, stream=None):
        """Clears gradient buffers (as splat_backward takes them) on ``stream``
        (default: the current stream), for a later call with grads_zeroed=True."""
        gp, gs, go, gd = grads
        n = gp.shape[0]
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        st = self.lib.tp_zero_gradients(ctypes.byref(self.cfg), n, _ptr(gp), _ptr(gs), _ptr(go), _ptr(gd),
                                        ctypes.c_void_p(s.cuda_stream))
        _lib.check("tp_zero_gradients", st)

    def camera_backward(self, pos, records, grad_pos, grad_size_w, out=None) -> torch.Tensor:
        """dL/d(fx, fy, cx, cy, R[0..8], t[0..2]) [16] float64, from this view's point gradients."""
        n = pos.shape[0]
        dev = self.device
        _need(pos, torch.float32, (n, 3), "pos", dev)
        _need(records, torch.float32, (n, 4), "records", dev)
        packed = _packed_pos_size(grad_pos, grad_size_w)
        if packed is None:
            _need(grad_pos, torch.float32, (n, 3), "grad_pos", dev)
            _need(grad_size_w, torch.float32, (n,), "grad_size_w", dev)
        if out is None:
            out = torch.empty(16, dtype=torch.float64, device=dev)
        st = self.lib.tp_camera_backward(ctypes.byref(self.cam), n, _ptr(pos), _ptr(records),
                                         _ptr(grad_pos if packed is None else packed),
                                         _ptr(grad_size_w if packed is None else None), _ptr(out), _stream(dev))
        _lib.check("tp_camera_backward", st)
        return out

    def merge(self, pyramid, out=None) -> torch.Tensor:
        """Merged layers [P, D] (the decoder's weight-free merge); rows [0, W H) are the image."""
        dev = self.device
        _need(pyramid, torch.float32, (self.P, self.D), "pyramid", dev)
        if out is None:
            out = torch.empty((self.P, self.D), dtype=torch.float32, device=dev)
        st = self.lib.tp_merge(ctypes.byref(self.cam), self.n_layers, self.D, _ptr(pyramid), _ptr(out), _stream(dev))
        _lib.check("tp_merge", st)
        return out

    def merge_backward(self, grad_image, out=None) -> torch.Tensor:
        """dL/dpyramid [P, D] from dL/d(merged image) [W H, D]."""
        dev = self.device
        _need(grad_image, torch.float32, (self.camera.width * self.camera.height, self.D), "grad_image", dev)
        if out is None:
            out = torch.empty((self.P, self.D), dtype=torch.float32, device=dev)
        st = self.lib.tp_merge_backward(ctypes.byref(self.cam), self.n_layers, self.D, _ptr(grad_image), _ptr(out),
                                        _stream(dev))
        _lib.check("tp_merge_backward", st)
        return out

    def status(self, ws) -> int:
        """Synchronises the current stream and returns the TP_FLAG_* bits of the frame."""
        flags = ctypes.c_int32(0)
        st = self.lib.tp_get_status(_ptr(ws), _stream(self.device), ctypes.byref(flags))
        if st == _lib.TP_ERR_CUDA or st == _lib.TP_ERR_INVALID_ARG:
            _lib.check("tp_get_status", st)
        return int(flags.value)

    # -- whole frames --------------------------------------------------------
    def render(self, pos, size_w, opacity, desc, store_lists=None, stats=False, ws=None) -> Frame:
        """Forward render: project, splat, blend."""
        n = pos.shape[0]
        if store_lists is None:
            store_lists = self.mode == _lib.TP_STORE_LISTS
        if ws is None:
            ws = self.new_workspace(n)
        records = self.project(pos, size_w, ws)
        self.splat_forward(records, opacity, ws)
        pyramid, kept, n_kept, t_final, n_frag = self.blend(records, opacity, desc, ws, store_lists, stats)
        return Frame(pyramid, records, ws, kept, n_kept, t_final, n_frag)

    def backward(self, frame: Frame, opacity, desc, grad_pyramid):
        """Gradients (pos, size_w, opacity, desc) of sum(grad_pyramid * pyramid) for a rendered frame."""
        use_lists = self.mode == _lib.TP_STORE_LISTS and frame.kept is not None
        return self.splat_backward(frame.records, opacity, desc, grad_pyramid.contiguous(), frame.workspace,
                                   frame.kept if use_lists else None, frame.n_kept if use_lists else None)


class TripsSplat(torch.autograd.Function):
    """pyramid = Phi(camera; pos, size_w, opacity, desc) with the hand-written adjoint."""

    @staticmethod
    def forward(ctx, pos, size_w, opacity, desc, renderer: Renderer):
        frame = renderer.render(pos.detach(), size_w.detach(), opacity.detach(), desc.detach())
        ctx.renderer = renderer
        ctx.frame = frame
        ctx.save_for_backward(opacity, desc)
        return frame.pyramid

    @staticmethod
    def backward(ctx, grad_pyramid):
        opacity, desc = ctx.saved_tensors
        gp, gs, go, gd = ctx.renderer.backward(ctx.frame, opacity.detach(), desc.detach(),
                                                grad_pyramid.to(torch.float32))
        ctx.frame = None
        return gp, gs, go, gd.to(desc.dtype), None


def splat(pos, size_w, opacity, desc, renderer: Renderer) -> torch.Tensor:
    """Differentiable trilinear point splatting into a [P, D] feature pyramid."""
    return TripsSplat.apply(pos, size_w, opacity, desc, renderer)


class BatchRenderer:
    """Several cameras rendered from one point cloud by the same launches.

    Each camera may have its own resolution and screen tile shape (``tiles``,
    one (tile_w, tile_h) per view, e.g. from :func:`autotune_tiles`).  The
    views' pyramids are concatenated in view order; ``view_offsets[v]`` is the
    first row of view v.  Gradients are those of the sum of the views' losses.
    """

    def __init__(self, cameras, n_layers: int, K: int = 16, D: int = 4, eps: float = 0.25,
                 desc_dtype=torch.float32, mode: str = "recompute", tiles=None, device=None, coarse: bool = False):
        self.lib = _lib.load()
        self.cameras = list(cameras)
        V = len(self.cameras)
        if not 1 <= V <= 16:
            raise ValueError("a batch holds 1 to 16 views")
        self.n_views = V
        self.cams = (_lib.tp_camera * V)(*[_lib.make_camera(c) for c in self.cameras])
        self.set_tiles(tiles)
        if desc_dtype not in _DTYPES:
            raise ValueError(f"descriptor dtype {desc_dtype} not supported")
        self.desc_dtype = desc_dtype
        self.mode = {"store": _lib.TP_STORE_LISTS, "recompute": _lib.TP_RECOMPUTE}[mode]
        self.coarse = bool(coarse)
        self.cfg = _lib.make_config(n_layers, K, D, eps, _DTYPES[desc_dtype], self.mode,
                                    flags=_lib.TP_COARSE_LAYERS if coarse else 0)
        self.n_layers, self.K, self.D = int(n_layers), int(K), int(D)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        offs = (ctypes.c_int64 * (V + 1))()
        P = self.lib.tp_batch_pixels(self.cams, V, n_layers, offs)
        if P < 0:
            raise ValueError("invalid cameras or layer count")
        self.P = int(P)
        self.view_offsets = [int(v) for v in offs]

    def set_tiles(self, tiles):
        if tiles is None:
            self.tiles = None
            self._tiles_c = None
        else:
            tiles = [tuple(int(a) for a in t) for t in tiles]
            if len(tiles) != self.n_views:
                raise ValueError("one tile shape per view")
            self.tiles = tiles
            self._tiles_c = (ctypes.c_int32 * (2 * self.n_views))(*[a for t in tiles for a in t])

    def _common(self):
        return ctypes.byref(self.cfg), self.cams, self._tiles_c, self.n_views

    def workspace_bytes(self, n: int, capacity: int = 0) -> int:
        b = self.lib.tp_batch_workspace_bytes(*self._common(), int(n), int(capacity))
        if b < 0:
            raise ValueError("invalid configuration for the workspace")
        return int(b)

    def new_workspace(self, n: int, capacity: int = 0) -> torch.Tensor:
        ws = torch.empty(self.workspace_bytes(n, capacity), dtype=torch.uint8, device=self.device)
        assert ws.data_ptr() % 256 == 0
        return ws

    def view(self, pyramid: torch.Tensor, v: int) -> torch.Tensor:
        """Rows of view v in a batched [P, ...] tensor."""
        return pyramid[self.view_offsets[v]:self.view_offsets[v + 1]]

    def project(self, pos, size_w, ws, records=None):
        n = pos.shape[0]
        _need(pos, torch.float32, (n, 3), "pos", self.device)
        _need(size_w, torch.float32, (n,), "size_w", self.device)
        if records is None:
            records = torch.empty((self.n_views, n, 4), dtype=torch.float32, device=self.device)
        st = self.lib.tp_batch_project(*self._common(), n, _ptr(pos), _ptr(size_w), _ptr(records), _ptr(ws),
                                       ws.numel(), _stream(self.device))
        _lib.check("tp_batch_project", st)
        return records

    def splat_forward(self, records, opacity, ws):
        n = records.shape[1]
        _need(opacity, torch.float32, (n,), "opacity", self.device)
        st = self.lib.tp_batch_splat_forward(*self._common(), n, _ptr(records), _ptr(opacity), _ptr(ws), ws.numel(),
                                             _stream(self.device))
        _lib.check("tp_batch_splat_forward", st)

    def blend(self, records, opacity, desc, ws, store_lists=False, stats=False, pyramid=None):
        n = records.shape[1]
        _need(records, torch.float32, (self.n_views, n, 4), "records", self.device)
        _need(opacity, torch.float32, (n,), "opacity", self.device)
        _need(desc, self.desc_dtype, (n, self.D), "desc", self.device)
        dev = self.device
        if pyramid is None:
            pyramid = torch.empty((self.P, self.D), dtype=torch.float32, device=dev)
        kept = n_kept = t_final = n_frag = None
        if store_lists or stats:
            kept = torch.empty((self.P, self.K), dtype=torch.int32, device=dev)
            n_kept = torch.empty((self.P,), dtype=torch.uint8, device=dev)
        if stats:
            t_final = torch.empty((self.P,), dtype=torch.float32, device=dev)
            n_frag = torch.empty((self.P,), dtype=torch.int32, device=dev)
        st = self.lib.tp_batch_blend(*self._common(), n, _ptr(records), _ptr(opacity), _ptr(desc), _ptr(pyramid),
                                     _ptr(kept), _ptr(n_kept), _ptr(t_final), _ptr(n_frag), _ptr(ws), ws.numel(),
                                     _stream(dev))
        _lib.check("tp_batch_blend", st)
        return pyramid, kept, n_kept, t_final, n_frag

    def splat_backward(self, records, opacity, desc, grad_pyramid, ws, kept=None, n_kept=None, grads=None):
        n = records.shape[1]
        dev = self.device
        _need(grad_pyramid, torch.float32, (self.P, self.D), "grad_pyramid", dev)
        (gp, gs, go, gd), out = _grad_buffers(n, self.D, dev, grads)
        st = self.lib.tp_batch_splat_backward(*self._common(), n, _ptr(records), _ptr(opacity), _ptr(desc),
                                              _ptr(kept), _ptr(n_kept), _ptr(grad_pyramid), _ptr(gp), _ptr(gs),
                                              _ptr(go), _ptr(gd), _ptr(ws), ws.numel(), _stream(dev))
        _lib.check("tp_batch_splat_backward", st)
        return out

    def splat_backward_cameras(self, pos, records, opacity, desc, grad_pyramid, ws, grads=None, grad_cameras=None):
        """Point gradients (recomputed lists) and every view's camera gradient
        dL/d(fx, fy, cx, cy, R[0..8], t[0..2]) [n_views, 16] float64 from one pass."""
        n = records.shape[1]
        dev = self.device
        _need(pos, torch.float32, (n, 3), "pos", dev)
        _need(grad_pyramid, torch.float32, (self.P, self.D), "grad_pyramid", dev)
        (gp, gs, go, gd), out = _grad_buffers(n, self.D, dev, grads)
        if grad_cameras is None:
            grad_cameras = torch.empty((self.n_views, 16), dtype=torch.float64, device=dev)
        st = self.lib.tp_batch_splat_backward_cameras(*self._common(), n, _ptr(pos), _ptr(records), _ptr(opacity),
                                                      _ptr(desc), _ptr(grad_pyramid), _ptr(gp), _ptr(gs), _ptr(go),
                                                      _ptr(gd), _ptr(grad_cameras), _ptr(ws), ws.numel(),
                                                      _stream(dev))
        _lib.check("tp_batch_splat_backward_cameras", st)
        return out, grad_cameras

    def status(self, ws) -> int:
        flags = ctypes.c_int32(0)
        st = self.lib.tp_get_status(_ptr(ws), _stream(self.device), ctypes.byref(flags))
        if st == _lib.TP_ERR_CUDA or st == _lib.TP_ERR_INVALID_ARG:
            _lib.check("tp_get_status", st)
        return int(flags.value)

    def render(self, pos, size_w, opacity, desc, store_lists=None, stats=False, ws=None) -> Frame:
        n = pos.shape[0]
        if store_lists is None:
            store_lists = self.mode == _lib.TP_STORE_LISTS
        if ws is None:
            ws = self.new_workspace(n)
        records = self.project(pos, size_w, ws)
        self.splat_forward(records, opacity, ws)
        pyramid, kept, n_kept, t_final, n_frag = self.blend(records, opacity, desc, ws, store_lists, stats)
        return Frame(pyramid, records, ws, kept, n_kept, t_final, n_frag)

    def backward(self, frame: Frame, opacity, desc, grad_pyramid):
        use_lists = self.mode == _lib.TP_STORE_LISTS and frame.kept is not None
        return self.splat_backward(frame.records, opacity, desc, grad_pyramid.contiguous(), frame.workspace,
                                   frame.kept if use_lists else None, frame.n_kept if use_lists else None)


# screen tiles the autotuners time: 64 to 512 pixels, square and wide shapes
TILE_CANDIDATES = ((16, 8), (16, 16), (32, 8), (8, 16), (8, 8), (32, 4), (16, 4), (24, 8), (16, 12), (32, 16),
                   (64, 4))


def autotune_tiles(cameras, n_layers, pos, size_w, opacity, desc, K=16, candidates=TILE_CANDIDATES, iters=3,
                   desc_dtype=torch.float32, device=None):
    """Per view, the screen tile shape with the fastest forward + backward.

    Every candidate renders the view alone (project, splat, blend, backward
    with a fixed upstream gradient) for ``iters`` timed iterations after one
    warm-up; the shape with the lowest median time wins.  Views of equal
    resolution are tuned once.  Returns (tiles, timings) where timings maps
    (width, height) to {tile: ms}.
    """
    n = pos.shape[0]
    D = desc.shape[1]
    best, timings = {}, {}
    for cam in cameras:
        res = (int(cam.width), int(cam.height))
        if res in best:
            continue
        times = {}
        for tile in candidates:
            try:
                r = Renderer(cam, n_layers, K=K, D=D, desc_dtype=desc_dtype, mode="recompute", tile=tile,
                             device=device)
                ws = r.new_workspace(n)
            except (ValueError, _lib.TripsError):
                continue
            G = torch.ones((r.P, D), dtype=torch.float32, device=r.device)
            rec = torch.empty((n, 4), dtype=torch.float32, device=r.device)
            pyr = torch.empty((r.P, D), dtype=torch.float32, device=r.device)
            grads = (torch.empty((n, 4), device=r.device), None,  # packed position/size rows
                     torch.empty((n,), device=r.device), torch.empty((n, D), device=r.device))
            ms = []
            try:
                for it in range(iters + 1):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    r.project(pos, size_w, ws, records=rec)
                    r.splat_forward(rec, opacity, ws)
                    r.blend(rec, opacity, desc, ws, pyramid=pyr)
                    r.splat_backward(rec, opacity, desc, G, ws, grads=grads)
                    e1.record()
                    torch.cuda.synchronize()
                    if it > 0:
                        ms.append(e0.elapsed_time(e1))
            except _lib.TripsError:
                continue
            times[tile] = sorted(ms)[len(ms) // 2]
            del ws, G, rec, pyr, grads
        if not times:
            raise RuntimeError(f"no tile shape works for {res}")
        best[res] = min(times, key=times.get)
        timings[res] = times
    return [best[(int(c.width), int(c.height))] for c in cameras], timings


def autotune_batch_tiles(cameras, n_layers, pos, size_w, opacity, desc, K=16, candidates=TILE_CANDIDATES, iters=3,
                         desc_dtype=torch.float32, device=None, start=None):
    """Screen tile shapes for a batch of views, tuned on the batch itself.

    A batch launch runs every tile CTA with the block of the batch's largest
    tile, so the shape that is fastest for a view rendered alone can slow the
    other views of the batch down.  Starting from ``start`` (default: 16 x 8
    for every view), each resolution in turn tries every candidate while the
    other resolutions keep their current shape, timing the whole batch step
    (project, splat, blend, backward with a fixed upstream gradient; median of
    ``iters`` after one warm-up), and keeps the fastest.  Returns (tiles,
    timings) where timings maps (width, height) to {tile: ms of the batch}.
    """
    cameras = list(cameras)
    n = pos.shape[0]
    D = desc.shape[1]
    res_of = [(int(c.width), int(c.height)) for c in cameras]
    groups = list(dict.fromkeys(res_of))
    current = dict(zip(res_of, start)) if start is not None else {r: (16, 8) for r in groups}
    buf = [None]

    def batch_ms(choice):
        tiles = [choice[r] for r in res_of]
        try:
            br = BatchRenderer(cameras, n_layers, K=K, D=D, desc_dtype=desc_dtype, mode="recompute", tiles=tiles,
                               device=device)
            need = br.workspace_bytes(n)
        except (ValueError, _lib.TripsError):
            return None
        if buf[0] is None or buf[0].numel() < need:
            buf[0] = None
            buf[0] = torch.empty(need, dtype=torch.uint8, device=br.device)
        ws = buf[0][:need]
        V = br.n_views
        G = torch.ones((br.P, D), dtype=torch.float32, device=br.device)
        rec = torch.empty((V, n, 4), dtype=torch.float32, device=br.device)
        pyr = torch.empty((br.P, D), dtype=torch.float32, device=br.device)
        grads = (torch.empty((n, 4), device=br.device), None,  # packed position/size rows
                 torch.empty((n,), device=br.device), torch.empty((n, D), device=br.device))
        ms = []
        try:
            for it in range(iters + 1):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                br.project(pos, size_w, ws, records=rec)
                br.splat_forward(rec, opacity, ws)
                br.blend(rec, opacity, desc, ws, pyramid=pyr)
                br.splat_backward(rec, opacity, desc, G, ws, grads=grads)
                e1.record()
                torch.cuda.synchronize()
                if it > 0:
                    ms.append(e0.elapsed_time(e1))
        except _lib.TripsError:
            return None
        return sorted(ms)[len(ms) // 2]

    timings = {}
    best_ms = batch_ms(current)
    if best_ms is None:
        raise RuntimeError("the starting tile shapes do not work for this batch")
    for res in groups:
        times = {current[res]: best_ms}
        for tile in candidates:
            tile = tuple(int(a) for a in tile)
            if tile in times:
                continue
            trial = dict(current)
            trial[res] = tile
            ms = batch_ms(trial)
            if ms is None:
                continue
            times[tile] = ms
        pick = min(times, key=times.get)
        current[res] = pick
        best_ms = times[pick]
        timings[res] = times
    buf[0] = None
    return [current[r] for r in res_of], timings


def init_point_sizes(pos: torch.Tensor, out: torch.Tensor | None = None, ws: torch.Tensor | None = None):
    """Initial world sizes [n]: mean distance to the 4 nearest other points (on the GPU)."""
    lib = _lib.load()
    if pos.dtype != torch.float32 or pos.dim() != 2 or pos.shape[1] != 3 or not pos.is_contiguous():
        raise ValueError("pos: expected contiguous float32 [n, 3]")
    n = pos.shape[0]
    dev = pos.device
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=dev)
    need = int(lib.tp_init_sizes_workspace_bytes(n))
    if need < 0:
        raise ValueError("too many points")
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    st = lib.tp_init_point_sizes(n, _ptr(pos), _ptr(out), _ptr(ws), ws.numel(), _stream(dev))
    _lib.check("tp_init_point_sizes", st)
    return out


def spatial_order(pos: torch.Tensor, ws: torch.Tensor | None = None) -> torch.Tensor:
    """Point indices [n] (int32 view of uint32) sorted by the Morton code of each
    point's cell in a 1024^3 grid over the cloud's bounding box (on the GPU).

    Relabel a cloud once with ``permute_rows`` (every per-point array with the
    same order) so that the points that meet in a screen tile are neighbours in
    memory; renders are the same up to the relabeling.
    """
    lib = _lib.load()
    if pos.dtype != torch.float32 or pos.dim() != 2 or pos.shape[1] != 3 or not pos.is_contiguous():
        raise ValueError("pos: expected contiguous float32 [n, 3]")
    n = pos.shape[0]
    dev = pos.device
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    need = int(lib.tp_spatial_order_workspace_bytes(n))
    if need < 0:
        raise ValueError("too many points")
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    st = lib.tp_spatial_order(n, _ptr(pos), _ptr(perm), _ptr(ws), ws.numel(), _stream(dev))
    _lib.check("tp_spatial_order", st)
    return perm


def permute_rows(t: torch.Tensor, perm: torch.Tensor) -> torch.Tensor:
    """A new tensor whose row k is row perm[k] of t (rows along dim 0; on the GPU)."""
    lib = _lib.load()
    if not t.is_contiguous() or t.dim() < 1:
        raise ValueError("t: expected a contiguous tensor")
    if perm.dtype != torch.int32 or perm.shape != (t.shape[0],) or not perm.is_contiguous():
        raise ValueError("perm: expected contiguous int32 [n]")
    out = torch.empty_like(t)
    n = t.shape[0]
    row_bytes = t.numel() // max(n, 1) * t.element_size() if n else 4
    st = lib.tp_permute_rows(n, row_bytes, _ptr(t), _ptr(perm), _ptr(out), _stream(t.device))
    _lib.check("tp_permute_rows", st)
    return out
