"""Pyramid merge (the decoder's weight-free layer merge) and its adjoint against the float64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import GRAD_RTOL, PYR_RTOL, assert_close_scaled, device, to_dev
from paper_2401_06003_gb300 import Renderer, scenes

pytestmark = pytest.mark.gpu

# A merged value is a float32 sum over the n layers of 4-tap bilinear sums of
# that layer's values; signed random inputs cancel, so its rounding error is
# bounded by about 3 n 2^-24 max|M| (1.4e-6 max|M| at n = 8), not by its own
# magnitude: the floor of the relative tolerance is 5e-2 of the layer's
# largest value (5e-7 max|M| at rtol 1e-5).
MERGE_FLOOR = 5e-2


def _renderer(W, H, n_layers, D):
    cam = scenes.camera_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), W, H)
    return Renderer(cam, n_layers, K=16, D=D, device=device())


@pytest.mark.parametrize("W,H,n,D", [(256, 192, 4, 4), (37, 22, 5, 3), (1, 1, 1, 4), (129, 65, 8, 16)])
def test_merge_matches_oracle(W, H, n, D):
    r = _renderer(W, H, n, D)
    rng = np.random.default_rng(W + H + n + D)
    P = rng.uniform(-1, 1, (r.P, D)).astype(np.float32)
    got = r.merge(to_dev(P)).cpu().numpy()
    ref = oracle.merge_pyramid(P, W, H, n)
    assert_close_scaled(got, ref, PYR_RTOL, floor=MERGE_FLOOR, name="merged layers",
                        segments=list(zip(r.layer_offsets[:-1], r.layer_offsets[1:])))
    # in place: the pyramid buffer receives the merged layers
    t = to_dev(P)
    r.merge(t, out=t)
    assert np.array_equal(t.cpu().numpy(), got)


@pytest.mark.parametrize("W,H,n,D", [(256, 192, 4, 4), (37, 22, 5, 3), (129, 65, 8, 16)])
def test_merge_backward_matches_oracle(W, H, n, D):
    r = _renderer(W, H, n, D)
    G = np.random.default_rng(W * H + D).uniform(-1, 1, (W * H, D)).astype(np.float32)
    got = r.merge_backward(to_dev(G)).cpu().numpy()
    ref = oracle.merge_pyramid_backward(G, W, H, n)
    assert_close_scaled(got, ref, GRAD_RTOL, name="merge adjoint", segments=list(zip(r.layer_offsets[:-1],
                                                                                      r.layer_offsets[1:])))
    # the image gradient may live in the first rows of the output
    buf = torch.zeros((r.P, D), device=device())
    buf[:W * H] = to_dev(G)
    r.merge_backward(buf[:W * H], out=buf)
    assert np.array_equal(buf.cpu().numpy(), got)


def test_merge_of_rendered_pyramid_1080p():
    """The merged image of the 6M-point frame (1920 x 1080, 8 layers)."""
    sc = scenes.make_config("ground6m_1080p")
    r = Renderer(sc.camera, sc.n_layers, K=sc.K, D=sc.D, device=device())
    fr = r.render(to_dev(sc.pos), to_dev(sc.size_w), to_dev(sc.opacity), to_dev(sc.desc))
    pyr = fr.pyramid.cpu().numpy()
    got = r.merge(fr.pyramid).cpu().numpy()
    ref = oracle.merge_pyramid(pyr, sc.camera.width, sc.camera.height, sc.n_layers)
    assert_close_scaled(got, ref, PYR_RTOL, name="merged 1080p", segments=list(zip(r.layer_offsets[:-1],
                                                                                    r.layer_offsets[1:])))
