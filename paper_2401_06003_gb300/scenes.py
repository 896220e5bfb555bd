"""Seeded synthetic scenes and cameras for trilinear point splatting.

This module only draws inputs: point positions, world sizes, descriptors,
opacities and pinhole cameras.  It holds none of the splatting arithmetic
(projection, layer choice, tap weights, blending), so both the CUDA path and
the CPU oracle can take their inputs from here without sharing method code.

The paper measures on Tanks&Temples, MipNeRF-360, Boat and Office point
clouds (Sec. 4.1).  None of those are available, so the generators below
stand in for them with scene-shaped clouds at the paper's point counts
(1.8M-72.5M points, Tab. "point_rend_eff"), resolutions (1080p, Sec. 4.4)
layer count (8, Tab. "layers_num") and descriptor width (4, Sec. 4.3).

Every generator uses ``numpy.random.default_rng(seed)`` (PCG64) and draws in
the order positions, sizes, descriptors, opacities.  Values are drawn in
float64 and stored as float32.

Camera convention (pinhole, OpenCV style): camera +z looks forward, +x is
image right, +y is image down.  ``R`` maps world to camera coordinates
(row-major), ``t`` is the translation, so ``X_c = R @ X_w + t``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Camera",
    "Scene",
    "look_at",
    "camera_at",
    "scene_uniform_cube",
    "scene_spheres",
    "scene_ground",
    "orbit_cameras",
    "make_config",
    "CONFIG_NAMES",
]


@dataclasses.dataclass
class Camera:
    """Pinhole camera: intrinsics (fx, fy, cx, cy), pose (R, t), image size."""

    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray  # [3, 3] float64, world -> camera, row-major
    t: np.ndarray  # [3] float64
    width: int
    height: int
    znear: float = 0.01

    def as_floats(self) -> np.ndarray:
        """The 17 camera floats in ABI order: fx, fy, cx, cy, R[9], t[3], znear."""
        return np.concatenate(
            [
                np.array([self.fx, self.fy, self.cx, self.cy], np.float64),
                np.asarray(self.R, np.float64).reshape(9),
                np.asarray(self.t, np.float64).reshape(3),
                np.array([self.znear], np.float64),
            ]
        ).astype(np.float32)


@dataclasses.dataclass
class Scene:
    """A point cloud with per-point attributes and one or more cameras."""

    name: str
    pos: np.ndarray  # [N, 3] float32 world positions
    size_w: np.ndarray  # [N] float32 world-space point size s_w
    desc: np.ndarray  # [N, D] float32 neural descriptors tau
    opacity: np.ndarray  # [N] float32 opacity alpha
    cameras: list
    n_layers: int
    K: int = 16

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def D(self) -> int:
        return int(self.desc.shape[1])

    @property
    def camera(self) -> Camera:
        return self.cameras[0]

    def subset(self, idx: np.ndarray, name: str | None = None) -> "Scene":
        idx = np.asarray(idx)
        return Scene(
            name=name or f"{self.name}[subset {idx.size}]",
            pos=np.ascontiguousarray(self.pos[idx]),
            size_w=np.ascontiguousarray(self.size_w[idx]),
            desc=np.ascontiguousarray(self.desc[idx]),
            opacity=np.ascontiguousarray(self.opacity[idx]),
            cameras=list(self.cameras),
            n_layers=self.n_layers,
            K=self.K,
        )


def look_at(eye, target, up=(0.0, 1.0, 0.0)):
    """World->camera rotation and translation for a camera at ``eye`` looking at ``target``.

    Camera +z points at the target, camera +y points along world -up (image
    rows grow downwards), camera +x = y x z completes a right-handed frame.
    """
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    up = np.asarray(up, np.float64)
    z = target - eye
    z /= np.linalg.norm(z)
    y = -up + np.dot(up, z) * z
    y /= np.linalg.norm(y)
    x = np.cross(y, z)
    R = np.stack([x, y, z], axis=0)
    t = -R @ eye
    return R, t


def camera_at(eye, target, width, height, up=(0.0, 1.0, 0.0), znear=0.01) -> Camera:
    """Pinhole camera with focal length f = height and the principal point at the centre."""
    R, t = look_at(eye, target, up)
    f = float(height)
    return Camera(f, f, width / 2.0, height / 2.0, R, t, int(width), int(height), znear)


def _uniform_sphere(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _finish(name, rng, pos, size_w, D, opacity_lo, cameras, n_layers, K):
    desc = rng.uniform(0.0, 1.0, size=(pos.shape[0], D))
    opacity = rng.uniform(opacity_lo, 1.0, size=pos.shape[0])
    return Scene(
        name=name,
        pos=np.ascontiguousarray(pos, dtype=np.float32),
        size_w=np.ascontiguousarray(size_w, dtype=np.float32),
        desc=np.ascontiguousarray(desc, dtype=np.float32),
        opacity=np.ascontiguousarray(opacity, dtype=np.float32),
        cameras=cameras,
        n_layers=n_layers,
        K=K,
    )


def scene_uniform_cube(n=20_000, seed=0, res=256, n_layers=4, D=4, K=16) -> Scene:
    """Points uniform in [-1,1]^3, sizes log-uniform in [1e-3, 5e-2], camera at z=-3, R=I."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-1.0, 1.0, size=(n, 3))
    size_w = np.exp(rng.uniform(math.log(1e-3), math.log(5e-2), size=n))
    cam = Camera(float(res), float(res), res / 2.0, res / 2.0, np.eye(3), np.array([0.0, 0.0, 3.0]), res, res)
    return _finish(f"cube{n}_{res}", rng, pos, size_w, D, 0.2, [cam], n_layers, K)


def scene_spheres(n=1_000_000, seed=0, width=1920, height=1080, n_layers=8, D=4, K=16,
                  n_spheres=50, clutter=0.10) -> Scene:
    """Points on the surfaces of random spheres plus uniform clutter; log-normal sizes.

    Sphere centres U[-1,1]^3, radii U(0.05,0.5); surface points are split over
    the spheres in proportion to their area.  Sizes s_w = 5e-3 * exp(0.7 N(0,1)).
    Camera at (0,0,-3) with R = I, f = height.
    """
    rng = np.random.default_rng(seed)
    n_clutter = int(round(n * clutter))
    n_surf = n - n_clutter
    centres = rng.uniform(-1.0, 1.0, size=(n_spheres, 3))
    radii = rng.uniform(0.05, 0.5, size=n_spheres)
    area = radii**2
    counts = np.floor(n_surf * area / area.sum()).astype(np.int64)
    counts[np.argmax(area)] += n_surf - counts.sum()
    which = np.repeat(np.arange(n_spheres), counts)
    surf = centres[which] + radii[which, None] * _uniform_sphere(rng, n_surf)
    clut = rng.uniform(-1.0, 1.0, size=(n_clutter, 3))
    pos = np.concatenate([surf, clut], axis=0)
    size_w = 5e-3 * np.exp(0.7 * rng.standard_normal(n))
    f = float(height)
    cam = Camera(f, f, width / 2.0, height / 2.0, np.eye(3), np.array([0.0, 0.0, 3.0]), width, height)
    return _finish(f"spheres{n}_{width}x{height}", rng, pos, size_w, D, 0.1, [cam], n_layers, K)


class _GradientNoise2D:
    """Improved gradient noise in 2D (Perlin 2002): quintic fade, hashed lattice gradients.

    The permutation is drawn from the scene's generator instead of a fixed
    table; the lattice gradients are the eight directions (+-1,+-1),
    (+-1,0), (0,+-1).
    """

    _G = np.array([[1, 1], [-1, 1], [1, -1], [-1, -1], [1, 0], [-1, 0], [0, 1], [0, -1]], np.float64)

    def __init__(self, rng):
        p = rng.permutation(256)
        self.perm = np.concatenate([p, p]).astype(np.int64)

    @staticmethod
    def _fade(t):
        return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)

    def _grad(self, h, dx, dy):
        g = self._G[h & 7]
        return g[..., 0] * dx + g[..., 1] * dy

    def __call__(self, x, y):
        xi = np.floor(x)
        yi = np.floor(y)
        fx = x - xi
        fy = y - yi
        X = xi.astype(np.int64) & 255
        Y = yi.astype(np.int64) & 255
        p = self.perm
        aa = p[p[X] + Y]
        ab = p[p[X] + Y + 1]
        ba = p[p[X + 1] + Y]
        bb = p[p[X + 1] + Y + 1]
        u = self._fade(fx)
        v = self._fade(fy)
        n00 = self._grad(aa, fx, fy)
        n10 = self._grad(ba, fx - 1.0, fy)
        n01 = self._grad(ab, fx, fy - 1.0)
        n11 = self._grad(bb, fx - 1.0, fy - 1.0)
        nx0 = n00 + u * (n10 - n00)
        nx1 = n01 + u * (n11 - n01)
        return nx0 + v * (nx1 - nx0)


def scene_ground(n=6_000_000, seed=0, width=1920, height=1080, n_layers=8, D=4, K=16,
                 n_clusters=32) -> Scene:
    """Scene-shaped cloud: noisy heightfield ground, Gaussian clusters, far background shell.

    60% on y = 0.2 * noise(x/4, z/4) over x,z in [-20,20] with N(0, 0.01)
    jitter; 20% in 32 Gaussian clusters (sigma ~ U(0.2,1)) centred on the
    ground; 20% uniform on a sphere of radius 50.  Sizes are Pareto
    (alpha = 2.5, x_min = 1e-3).  Opacity U(0.1,1).  Camera at (0,1.7,-12)
    looking at (0,0.5,0), world up +y.
    """
    rng = np.random.default_rng(seed)
    noise = _GradientNoise2D(rng)
    n_ground = int(round(0.6 * n))
    n_clu = int(round(0.2 * n))
    n_shell = n - n_ground - n_clu

    gx = rng.uniform(-20.0, 20.0, size=n_ground)
    gz = rng.uniform(-20.0, 20.0, size=n_ground)
    gy = 0.2 * noise(gx / 4.0, gz / 4.0)
    ground = np.stack([gx, gy, gz], axis=1) + rng.normal(0.0, 0.01, size=(n_ground, 3))

    sig = rng.uniform(0.2, 1.0, size=n_clusters)
    cx = rng.uniform(-20.0, 20.0, size=n_clusters)
    cz = rng.uniform(-20.0, 20.0, size=n_clusters)
    cy = 0.2 * noise(cx / 4.0, cz / 4.0)
    counts = np.full(n_clusters, n_clu // n_clusters, np.int64)
    counts[: n_clu - counts.sum()] += 1
    which = np.repeat(np.arange(n_clusters), counts)
    centres = np.stack([cx, cy, cz], axis=1)
    clusters = centres[which] + sig[which, None] * rng.standard_normal((n_clu, 3))

    shell = 50.0 * _uniform_sphere(rng, n_shell)
    pos = np.concatenate([ground, clusters, shell], axis=0)
    size_w = 1e-3 * (1.0 + rng.pareto(2.5, size=n))
    cam = camera_at((0.0, 1.7, -12.0), (0.0, 0.5, 0.0), width, height)
    return _finish(f"ground{n}_{width}x{height}", rng, pos, size_w, D, 0.1, [cam], n_layers, K)


ORBIT_RESOLUTIONS = ((640, 480), (1280, 720), (1920, 1080), (2560, 1440))


def orbit_cameras(n_views=16, seed=1, radius=12.0, height=1.7, target=(0.0, 0.5, 0.0)):
    """Cameras on a circular orbit, each with a resolution drawn from ORBIT_RESOLUTIONS.

    View k sits at azimuth 2*pi*k/n_views; view 0 is the single camera of
    :func:`scene_ground`.  The resolutions use their own generator (``seed``)
    so the point cloud is unchanged.
    """
    rng = np.random.default_rng(seed)
    picks = rng.integers(0, len(ORBIT_RESOLUTIONS), size=n_views)
    cams = []
    for k in range(n_views):
        th = 2.0 * math.pi * k / n_views
        eye = (radius * math.sin(th), height, -radius * math.cos(th))
        w, h = ORBIT_RESOLUTIONS[int(picks[k])]
        cams.append(camera_at(eye, target, w, h))
    return cams


CONFIG_NAMES = ("cube20k_256", "spheres1m_1080p", "ground6m_1080p", "ground6m_orbit16", "ground10m_4k_bf16")


def make_config(name: str, n: int | None = None, seed: int = 0) -> Scene:
    """The five benchmark workloads by name; ``n`` overrides the point count."""
    if name == "cube20k_256":
        return scene_uniform_cube(n=n or 20_000, seed=seed)
    if name == "spheres1m_1080p":
        return scene_spheres(n=n or 1_000_000, seed=seed)
    if name == "ground6m_1080p":
        return scene_ground(n=n or 6_000_000, seed=seed)
    if name == "ground6m_orbit16":
        s = scene_ground(n=n or 6_000_000, seed=seed)
        s.cameras = orbit_cameras()
        s.name = f"ground{s.n}_orbit16"
        return s
    if name == "ground10m_4k_bf16":
        return scene_ground(n=n or 10_000_000, seed=seed, width=3840, height=2160, n_layers=10, D=16)
    raise KeyError(name)
