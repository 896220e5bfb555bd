"""Camera adjoint (intrinsics and pose) against the float64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import GRAD_RTOL, assert_close_scaled, device, to_dev
from paper_2401_06003_gb300 import Renderer, TripsError, scenes

pytestmark = pytest.mark.gpu

GROUPS = [(0, 4), (4, 13), (13, 16)]  # intrinsics, rotation, translation: each scaled by its own max


def _camera_grad(sc, cam, mode, seed):
    r = Renderer(cam, sc.n_layers, K=sc.K, D=sc.D, mode=mode, device=device())
    pos, sw, op, desc = to_dev(sc.pos), to_dev(sc.size_w), to_dev(sc.opacity), to_dev(sc.desc)
    fr = r.render(pos, sw, op, desc)
    G = np.random.default_rng(seed).uniform(-1, 1, (r.P, sc.D)).astype(np.float32)
    gp, gsw, _, _ = r.splat_backward(fr.records, op, desc, to_dev(G), fr.workspace, kept=fr.kept,
                                     n_kept=fr.n_kept)
    got = r.camera_backward(pos, fr.records, gp, gsw).cpu().numpy()
    assert r.status(fr.workspace) == 0
    s = sc.subset(np.arange(sc.n))
    s.cameras = [cam]
    ref = oracle.Frame.from_scene(s).camera_backward(G.astype(np.float64))
    return got, ref


@pytest.mark.parametrize("mode", ["recompute", "store"])
def test_camera_adjoint_cube(mode):
    sc = scenes.make_config("cube20k_256")
    cam = scenes.camera_at((0.9, 0.6, -2.6), (0.05, -0.1, 0.0), 256, 192)
    got, ref = _camera_grad(sc, cam, mode, seed=11)
    assert_close_scaled(got, ref, GRAD_RTOL, name="camera gradient", segments=GROUPS)


def test_camera_adjoint_spheres1m_1080p():
    sc = scenes.make_config("spheres1m_1080p")
    got, ref = _camera_grad(sc, sc.cameras[0], "recompute", seed=12)
    assert_close_scaled(got, ref, GRAD_RTOL, name="camera gradient 1M", segments=GROUPS)


def test_camera_adjoint_no_visible_points_is_zero():
    sc = scenes.scene_uniform_cube(n=500, seed=2, res=64)
    cam = scenes.camera_at((0.0, 0.0, 3.0), (0.0, 0.0, 6.0), 64, 64)  # looking away from the cloud
    got, _ = _camera_grad(sc, cam, "recompute", seed=13)
    assert np.all(got == 0.0)


def test_camera_adjoint_rejects_singular_rotation():
    sc = scenes.scene_uniform_cube(n=100, seed=2, res=64)
    cam = scenes.camera_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 64, 64)
    r = Renderer(cam, sc.n_layers, K=sc.K, D=sc.D, device=device())
    r.cam.R = (type(r.cam.R))(*([0.0] * 9))
    z = torch.zeros((sc.n, 3), device=device())
    with pytest.raises(TripsError) as e:
        r.camera_backward(z, torch.zeros((sc.n, 4), device=device()), z, torch.zeros(sc.n, device=device()))
    assert e.value.status == 1
