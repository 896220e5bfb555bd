"""Pins of the oracle's pyramid merge (Sec. 3.3, weight-free form) and its adjoint."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("Hc,Wc,odd_h,odd_w", [(1, 1, 0, 0), (3, 5, 1, 0), (4, 4, 0, 1), (7, 2, 1, 1), (6, 9, 0, 0)])
def test_upsample_is_torch_bilinear(Hc, Wc, odd_h, odd_w):
    """up2 is bilinear interpolation at scale 2 with half-pixel centres (the
    library routine, computed in float64), cropped when the finer layer is odd."""
    rng = np.random.default_rng(Hc * 31 + Wc)
    C = rng.uniform(-1, 1, (Hc, Wc, 3))
    H, W = 2 * Hc - odd_h, 2 * Wc - odd_w
    ref = torch.nn.functional.interpolate(torch.from_numpy(C).permute(2, 0, 1)[None], scale_factor=2,
                                          mode="bilinear", align_corners=False)[0].permute(1, 2, 0).numpy()
    np.testing.assert_allclose(oracle.upsample2(C, H, W), ref[:H, :W], rtol=0, atol=1e-14)


def test_constant_layers_sum():
    """Bilinear weights sum to one, so constant layers merge to the sum of the constants."""
    W, H, n = 37, 22, 5
    off, _, _ = oracle.pyramid_layout(W, H, n)
    c = np.array([0.5, -2.0, 3.25, 1.0, 7.0])
    P = np.zeros((off[-1], 2))
    for L in range(n):
        P[off[L]:off[L + 1]] = c[L]
    M = oracle.merge_pyramid(P, W, H, n)
    np.testing.assert_allclose(M[:W * H], c.sum(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(M[off[n - 1]:], c[n - 1], rtol=0, atol=0)


def test_single_layer_is_identity_and_top_layer_passes_through():
    W, H = 9, 7
    P = np.random.default_rng(1).uniform(size=(W * H, 4))
    np.testing.assert_array_equal(oracle.merge_pyramid(P, W, H, 1), P)


@pytest.mark.parametrize("W,H,n", [(40, 30, 4), (33, 17, 5), (8, 8, 4)])
def test_adjoint_dot_product(W, H, n):
    """<merge(P)_image, G> == <P, merge_backward(G)> for random P and G."""
    rng = np.random.default_rng(W * H + n)
    off, _, _ = oracle.pyramid_layout(W, H, n)
    P = rng.uniform(-1, 1, (off[-1], 3))
    G = rng.uniform(-1, 1, (W * H, 3))
    lhs = float((oracle.merge_pyramid(P, W, H, n)[:W * H] * G).sum())
    rhs = float((P * oracle.merge_pyramid_backward(G, W, H, n)).sum())
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


def test_merge_is_the_recursion():
    """M_L = P_L + up2(M_{L+1}) layer by layer (spelled out for three layers)."""
    W, H, n = 12, 10, 3
    off, ws, hs = oracle.pyramid_layout(W, H, n)
    rng = np.random.default_rng(5)
    P = rng.uniform(size=(off[-1], 2))
    lay = [P[off[L]:off[L + 1]].reshape(hs[L], ws[L], 2) for L in range(n)]
    m2 = lay[2]
    m1 = lay[1] + oracle.upsample2(m2, hs[1], ws[1])
    m0 = lay[0] + oracle.upsample2(m1, hs[0], ws[0])
    np.testing.assert_allclose(oracle.merge_pyramid(P, W, H, n)[:W * H], m0.reshape(-1, 2), rtol=0, atol=1e-14)
