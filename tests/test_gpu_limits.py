"""The library's documented maxima against the float64 oracle: descriptor width
64, 16 pyramid layers, an image 32768 pixels wide."""
import numpy as np
import pytest

import oracle
from gpu_helpers import GRAD_RTOL, assert_close_scaled, compare_forward, compare_records, gpu_frame, to_dev
from paper_2401_06003_gb300 import Renderer, scenes

pytestmark = pytest.mark.gpu


def _scene(n, W, H, n_layers, D, K=16, seed=21, eye=(0.3, 0.2, -3.0)):
    sc = scenes.scene_uniform_cube(n=n, seed=seed, res=64)
    rng = np.random.default_rng(seed + 7)
    # non-negative descriptors as in the workloads' recipe: the pyramid's 1e-5
    # tolerance assumes blended sums that do not cancel
    sc.desc = rng.uniform(0, 1, (n, D)).astype(np.float32)
    sc.cameras = [scenes.camera_at(eye, (0.0, 0.0, 0.0), W, H)]
    sc.n_layers, sc.K = n_layers, K
    return sc


def _check(sc, backward=True):
    r, fr, _, out = gpu_frame(sc, mode="recompute")
    ofr = oracle.Frame.from_scene(sc)
    compare_records(out["records"], ofr)
    compare_forward(out, ofr.render(), r.layer_offsets, name=f"{sc.cameras[0].width}x{sc.cameras[0].height}")
    if backward:
        G = np.random.default_rng(3).uniform(-1, 1, (r.P, sc.D)).astype(np.float32)
        gp, gs, go, gd = r.splat_backward(fr.records, to_dev(sc.opacity), to_dev(sc.desc), to_dev(G), fr.workspace)
        ref = ofr.backward(G.astype(np.float64))
        for got, k in ((gp, "pos"), (gs, "size_w"), (go, "opacity"), (gd, "desc")):
            assert_close_scaled(got.cpu().numpy().reshape(sc.n, -1), ref[k].reshape(sc.n, -1), GRAD_RTOL,
                                name=f"grad {k}")


def test_descriptor_width_64():
    _check(_scene(3000, 96, 64, 4, D=64))


def test_sixteen_layers():
    # a 600 x 300 image has layers down to 1 x 1 well before the 16th
    _check(_scene(4000, 600, 300, 16, D=4))


def test_widest_image():
    # 32768 x 2 pixels (layer widths 32768 ... 1024, heights 2 then 1); the
    # cube spans 8000 columns and sizes reach past the coarsest layer (clamped)
    sc = _scene(3000, 64, 64, 6, D=4)
    sc.cameras = [scenes.Camera(8000.0, 0.5, 16384.0, 1.0, np.eye(3), np.array([0.0, 0.0, 3.0]), 32768, 2)]
    _check(sc)
