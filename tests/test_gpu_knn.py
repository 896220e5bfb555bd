"""Point-size initialisation (Sec. 3.6) on the GPU against the float64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import PYR_RTOL, assert_close_scaled, device, to_dev
from paper_2401_06003_gb300 import init_point_sizes, scenes

pytestmark = pytest.mark.gpu
pytest.importorskip("scipy")


def _gpu(pos):
    return init_point_sizes(to_dev(pos)).cpu().numpy()


def test_cube20k():
    sc = scenes.make_config("cube20k_256")
    assert_close_scaled(_gpu(sc.pos), oracle.init_point_sizes(sc.pos), PYR_RTOL, name="sizes cube")


def test_clusters_duplicates_and_nonfinite():
    rng = np.random.default_rng(3)
    centres = rng.uniform(-50, 50, (20, 3))
    scale = np.exp(rng.uniform(np.log(1e-3), np.log(2.0), 20))  # densities over three decades
    lab = rng.integers(0, 20, 8000)
    pos = (centres[lab] + rng.normal(size=(8000, 3)) * scale[lab, None]).astype(np.float32)
    pos[100:150] = pos[200:250]        # duplicates at distance 0
    pos[7000:7010] = pos[7010]         # eleven copies of one point
    pos[5, 1] = np.nan
    pos[6, 2] = np.inf
    got = _gpu(pos)
    ref = oracle.init_point_sizes(pos)
    assert got[5] == 0 and got[6] == 0
    assert np.all(got[7000:7011] == 0)
    assert_close_scaled(got, ref, PYR_RTOL, name="sizes clusters")


def test_tiny_inputs():
    assert _gpu(np.zeros((1, 3), np.float32)).tolist() == [0.0]
    np.testing.assert_allclose(_gpu(np.array([[0, 0, 0], [3, 4, 0]], np.float32)), [5.0, 5.0], rtol=1e-6)
    pos = np.array([[0, 0, 0], [1, 0, 0], [0, 2, 0]], np.float32)
    np.testing.assert_allclose(_gpu(pos), oracle.init_point_sizes(pos), rtol=1e-6)
    assert init_point_sizes(torch.zeros((0, 3), device=device())).numel() == 0


def test_lattice_closed_form():
    h = 0.37
    g = np.arange(9, dtype=np.float32) * np.float32(h)
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    s = _gpu(pos).reshape(9, 9, 9)
    np.testing.assert_allclose(s[1:-1, 1:-1, 1:-1], h, rtol=1e-6)
    np.testing.assert_allclose(s[0, 0, 0], (3 * h + h * math.sqrt(2)) / 4, rtol=1e-6)


def test_ground6m_sampled():
    """The 6M-point cloud (a dense ground, clusters and a sparse far shell): 20k sampled points."""
    sc = scenes.make_config("ground6m_1080p")
    got = _gpu(sc.pos)
    pts = np.random.default_rng(9).choice(sc.n, 20000, replace=False)
    ref = oracle.init_point_sizes(sc.pos, points=pts)
    assert_close_scaled(got[pts], ref, PYR_RTOL, name="sizes ground6m")
    assert np.all(got > 0)
