"""CPU oracle for trilinear point splatting (float64; test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The product path (the CUDA
library and its Python binding) never does.

The arithmetic lives in ``trips_oracle.c`` (plain C, built with gcc); this
module compiles it on first use and wraps it with ctypes.  Paper references:
projection Sec. 3.1 Eq. 2, weights Eq. 3-5, lists and blending Sec. 3.2
Eq. 6-7, list cap and stored sorted lists Sec. 3.6.

Parity status per function (what pins each one is in ``tests/test_oracle*``):
  projection, layer choice, tap weights   pinned (closed forms, brute force)
  fragment lists / K cap / order          pinned (brute force on tiny inputs)
  blending                                pinned (closed forms, brute force)
  adjoint                                 pinned (central finite differences)
  camera adjoint                          pinned (central finite differences of the camera)
  pyramid merge and its adjoint           pinned (torch bilinear interpolation, closed
                                          forms, dot-product test)
  point-size initialisation               pinned (brute force, lattice closed forms)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trips_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.orc_pyramid_layout.restype = i64
        lib.orc_pyramid_layout.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P]
        lib.orc_frame_build.restype = P
        lib.orc_frame_build.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dbl,
                                        ctypes.c_int, i64, P, P, P, P, ctypes.c_int, i64, P, i64, P, ctypes.c_int]
        lib.orc_frame_free.argtypes = [P]
        for name in ("orc_frame_num_pixels", "orc_frame_num_fragments", "orc_frame_num_bad"):
            getattr(lib, name).restype = i64
            getattr(lib, name).argtypes = [P]
        lib.orc_frame_pixels.argtypes = [P, P]
        lib.orc_frame_records.argtypes = [P, P, P]
        lib.orc_frame_fragments.argtypes = [P, P, P, P, P]
        lib.orc_frame_render.argtypes = [P, P, P, P, P, P]
        lib.orc_frame_backward.argtypes = [P, P, P, P, P, P, P]
        lib.orc_frame_camera_backward.argtypes = [P, P, P]
        lib.orc_frame_fd.restype = ctypes.c_int
        lib.orc_frame_fd.argtypes = [P, P, i64, P, dbl, dbl, dbl, dbl, P, P]
        del i32
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def pyramid_layout(width: int, height: int, n_layers: int):
    """(offsets [n_layers+1], widths, heights) of the concatenated pyramid."""
    lib = _load()
    off = np.zeros(n_layers + 1, np.int64)
    w = np.zeros(n_layers, np.int32)
    h = np.zeros(n_layers, np.int32)
    lib.orc_pyramid_layout(int(width), int(height), int(n_layers), _ptr(off), _ptr(w), _ptr(h))
    return off, w, h


class Frame:
    """All fragment lists of one rendered view (or of a subset of its pixels).

    ``prec32=True`` takes the projection, and every integer decision that
    follows from it, in float32 with the operation order the CUDA kernels
    use; ``prec32=False`` is the all-float64 reading (needed for finite
    differences).  Weights, blending and the adjoint are float64 either way.
    ``coarse=True`` adds the coarse-layer inclusion of Sec. 3.6: a pixel's
    list also holds the fragments of the coarser-layer pixels that contain it
    (reading R24 in the C source).
    """

    def __init__(self, cam_floats, width, height, n_layers, K, pos, size_w, opacity, desc,
                 eps=0.25, prec32=True, pixels=None, points=None, coarse=False):
        self._lib = _load()
        self.pos = np.ascontiguousarray(pos, np.float32)
        self.size_w = np.ascontiguousarray(size_w, np.float32)
        self.opacity = np.ascontiguousarray(opacity, np.float32)
        self.desc = np.ascontiguousarray(desc, np.float32)
        self.cam = np.ascontiguousarray(cam_floats, np.float32)
        assert self.cam.shape == (17,)
        self.n = int(self.pos.shape[0])
        self.D = int(self.desc.shape[1]) if self.desc.ndim == 2 else 1
        self.K = int(K)
        self.n_layers = int(n_layers)
        self.width, self.height = int(width), int(height)
        self.prec32 = bool(prec32)
        pix = None if pixels is None else np.ascontiguousarray(np.unique(np.asarray(pixels, np.int64)))
        pts = None if points is None else np.ascontiguousarray(np.asarray(points, np.int64))
        self._h = self._lib.orc_frame_build(
            _ptr(self.cam), self.width, self.height, self.n_layers, self.K, float(eps), self.D,
            self.n, _ptr(self.pos), _ptr(self.size_w), _ptr(self.opacity), _ptr(self.desc),
            int(self.prec32), 0 if pix is None else pix.size, _ptr(pix), 0 if pts is None else pts.size, _ptr(pts),
            int(bool(coarse)))
        if not self._h:
            raise MemoryError("oracle frame build failed")
        self.n_pix = int(self._lib.orc_frame_num_pixels(self._h))
        self.n_frag = int(self._lib.orc_frame_num_fragments(self._h))
        self.n_bad = int(self._lib.orc_frame_num_bad(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_frame_free(h)
            self._h = None

    @classmethod
    def from_scene(cls, scene, view=0, prec32=True, pixels=None, points=None, desc=None, coarse=False):
        cam = scene.cameras[view]
        return cls(cam.as_floats(), cam.width, cam.height, scene.n_layers, scene.K, scene.pos, scene.size_w,
                   scene.opacity, scene.desc if desc is None else desc, prec32=prec32, pixels=pixels, points=points,
                   coarse=coarse)

    def pixels(self) -> np.ndarray:
        out = np.zeros(self.n_pix, np.int64)
        self._lib.orc_frame_pixels(self._h, _ptr(out))
        return out

    def records(self):
        """Projected (x, y, z, s) [n,4] float64 and visibility [n] int8."""
        xyzs = np.zeros((self.n, 4), np.float64)
        vis = np.zeros(self.n, np.int8)
        self._lib.orc_frame_records(self._h, _ptr(xyzs), _ptr(vis))
        return xyzs, vis

    def fragments(self):
        """Every fragment in sorted (pixel, z, i) order: pixel, z, point, beta*iota."""
        n = self.n_frag
        pix = np.zeros(n, np.int64)
        z = np.zeros(n, np.float64)
        idx = np.zeros(n, np.int32)
        w = np.zeros(n, np.float64)
        self._lib.orc_frame_fragments(self._h, _ptr(pix), _ptr(z), _ptr(idx), _ptr(w))
        return pix, z, idx, w

    def render(self):
        """Blend every frame pixel: dict of pyramid, kept, n_kept, t_final, n_frag."""
        P, D, K = self.n_pix, self.D, self.K
        out = dict(
            pyramid=np.zeros((P, D), np.float64),
            kept=np.zeros((P, K), np.int32),
            n_kept=np.zeros(P, np.int32),
            t_final=np.zeros(P, np.float64),
            n_frag=np.zeros(P, np.int32),
        )
        self._lib.orc_frame_render(self._h, _ptr(out["pyramid"]), _ptr(out["kept"]), _ptr(out["n_kept"]),
                                   _ptr(out["t_final"]), _ptr(out["n_frag"]))
        return out

    def backward(self, G):
        """Gradients of sum(G * C) over the frame's pixels w.r.t. all point inputs."""
        G = np.ascontiguousarray(G, np.float64).reshape(self.n_pix, self.D)
        n, D = self.n, self.D
        out = dict(
            pos=np.zeros((n, 3), np.float64),
            size_w=np.zeros(n, np.float64),
            opacity=np.zeros(n, np.float64),
            desc=np.zeros((n, D), np.float64),
            screen=np.zeros((n, 3), np.float64),
        )
        self._lib.orc_frame_backward(self._h, _ptr(G), _ptr(out["pos"]), _ptr(out["size_w"]),
                                     _ptr(out["opacity"]), _ptr(out["desc"]), _ptr(out["screen"]))
        return out

    def camera_backward(self, G):
        """dL/d(fx, fy, cx, cy, R[0..8], t[0..2]) of sum(G * C) over the frame's pixels [16]."""
        G = np.ascontiguousarray(G, np.float64).reshape(self.n_pix, self.D)
        out = np.zeros(16, np.float64)
        self._lib.orc_frame_camera_backward(self._h, _ptr(G), _ptr(out))
        return out

    def finite_differences(self, G, points, h_pos=1e-6, h_sw_rel=1e-6, h_alpha=1e-6, h_desc=1e-3):
        """Local central differences for the given points: (fd [m, 5+D], valid [m, 5+D]).

        Columns: X, Y, Z, s_w, alpha, desc[0..D).  In a ``prec32`` frame the
        differences are float64 changes around the frame's float32
        screen-space state (the state its integer decisions were taken at).
        """
        G = np.ascontiguousarray(G, np.float64).reshape(self.n_pix, self.D)
        pts = np.ascontiguousarray(np.asarray(points, np.int64))
        fd = np.zeros((pts.size, 5 + self.D), np.float64)
        valid = np.zeros((pts.size, 5 + self.D), np.int8)
        rc = self._lib.orc_frame_fd(self._h, _ptr(G), pts.size, _ptr(pts), h_pos, h_sw_rel, h_alpha, h_desc,
                                    _ptr(fd), _ptr(valid))
        if rc != 0:
            raise RuntimeError(f"oracle finite differences failed ({rc})")
        return fd, valid.astype(bool)


# ---------------------------------------------------------------------------
# Pyramid merge: the fixed (weight-free) form of the decoder's layer merge
# (Sec. 3.3: every layer but the finest is upsampled bilinearly and merged
# with the next finer one).  Merging is a sum:
#   M_{n-1} = P_{n-1},   M_L = P_L + up2(M_{L+1}),
# and up2 samples layer L+1 at the layer-L pixel centres: pixel j of layer L
# sits at (j + 0.5) 2^L, i.e. at r = (j + 0.5)/2 - 0.5 in layer L+1 units,
# clamped to r >= 0; taps x0 = floor(r) and min(x0 + 1, W_{L+1} - 1) with
# weights 1 - (r - x0) and r - x0.  M_0 is the merged full-resolution image.
# ---------------------------------------------------------------------------

def _up2_axis(n_out, n_in):
    r = np.maximum((np.arange(n_out, dtype=np.float64) + 0.5) / 2.0 - 0.5, 0.0)
    x0 = np.floor(r).astype(np.int64)
    x1 = np.minimum(x0 + 1, n_in - 1)
    return x0, x1, r - x0


def upsample2(C, H, W):
    """Bilinear x2 upsampling of C [Hc, Wc, D] to [H, W, D] (H <= 2 Hc, W <= 2 Wc)."""
    C = np.asarray(C, np.float64)
    y0, y1, ly = _up2_axis(H, C.shape[0])
    x0, x1, lx = _up2_axis(W, C.shape[1])
    lx = lx[None, :, None]
    top = C[y0][:, x0] * (1.0 - lx) + C[y0][:, x1] * lx
    bot = C[y1][:, x0] * (1.0 - lx) + C[y1][:, x1] * lx
    return top * (1.0 - ly)[:, None, None] + bot * ly[:, None, None]


def upsample2_adjoint(G, Hc, Wc):
    """Transpose of upsample2: G [H, W, D] -> [Hc, Wc, D]."""
    G = np.asarray(G, np.float64)
    H, W, D = G.shape
    y0, y1, ly = _up2_axis(H, Hc)
    x0, x1, lx = _up2_axis(W, Wc)
    out = np.zeros((Hc, Wc, D), np.float64)
    for yy, wy in ((y0, 1.0 - ly), (y1, ly)):
        for xx, wx in ((x0, 1.0 - lx), (x1, lx)):
            np.add.at(out, (yy[:, None], xx[None, :]), G * (wy[:, None] * wx[None, :])[:, :, None])
    return out


def merge_pyramid(pyramid, width, height, n_layers):
    """Merged layers M [P, D] in the pyramid's layout; rows [0, W H) are the image."""
    off, ws, hs = pyramid_layout(width, height, n_layers)
    P = np.asarray(pyramid, np.float64)
    D = P.shape[1]
    M = np.zeros_like(P)
    for L in range(n_layers - 1, -1, -1):
        layer = P[off[L]:off[L + 1]].reshape(hs[L], ws[L], D)
        if L < n_layers - 1:
            coarse = M[off[L + 1]:off[L + 2]].reshape(hs[L + 1], ws[L + 1], D)
            layer = layer + upsample2(coarse, hs[L], ws[L])
        M[off[L]:off[L + 1]] = layer.reshape(-1, D)
    return M


def merge_pyramid_backward(grad_image, width, height, n_layers):
    """dL/dP [P, D] from dL/d(image) [W H, D]: dL/dP_L = dL/dM_L, dL/dM_{L+1} = up2^T dL/dM_L."""
    off, ws, hs = pyramid_layout(width, height, n_layers)
    g = np.asarray(grad_image, np.float64)
    D = g.shape[1]
    out = np.zeros((int(off[-1]), D), np.float64)
    gm = g.reshape(hs[0], ws[0], D)
    for L in range(n_layers):
        out[off[L]:off[L + 1]] = gm.reshape(-1, D)
        if L + 1 < n_layers:
            gm = upsample2_adjoint(gm, hs[L + 1], ws[L + 1])
    return out


# ---------------------------------------------------------------------------
# Point-size initialisation (Sec. 3.6): each point's initial world size is
# the mean distance to its four nearest other points.  A point's own index is
# never its neighbour; duplicates at distance 0 are.  With fewer than five
# points the mean runs over the n - 1 others (0 for a single point).  Points
# with a non-finite coordinate are nobody's neighbour and get size 0.
# ---------------------------------------------------------------------------

def init_point_sizes(pos, k=4, points=None):
    """Mean distance to the k nearest other points, float64 (KD-tree query).

    Returns sizes for every point, or for the indices in ``points`` only."""
    from scipy.spatial import cKDTree

    P = np.asarray(pos, np.float64)
    n = P.shape[0]
    sel = np.arange(n) if points is None else np.asarray(points, np.int64)
    out = np.zeros(sel.size, np.float64)
    ok = np.isfinite(P).all(axis=1)
    idx = np.nonzero(ok)[0]
    m = idx.size
    if m < 2:
        return out
    kk = min(k, m - 1)
    tree = cKDTree(P[idx])
    local = np.full(n, -1, np.int64)
    local[idx] = np.arange(m)
    qsel = np.nonzero(ok[sel])[0]
    dist, nb = tree.query(P[sel[qsel]], k=kk + 1)
    dist = dist.reshape(qsel.size, kk + 1)
    nb = nb.reshape(qsel.size, kk + 1)
    for r, q in enumerate(qsel):
        own = np.nonzero(nb[r] == local[sel[q]])[0]
        keep = np.delete(dist[r], own[0] if own.size else kk)  # drop the point itself, else the farthest
        out[q] = keep.mean()
    return out

