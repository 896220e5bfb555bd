"""Pins of the oracle's point-size initialisation (Sec. 3.6: mean distance to
the four nearest neighbours)."""
import math

import numpy as np
import pytest

import oracle

pytest.importorskip("scipy")


def _brute(pos, k=4):
    """Every pair's distance, sorted per point (small inputs only)."""
    P = np.asarray(pos, np.float64)
    n = P.shape[0]
    ok = np.isfinite(P).all(axis=1)
    out = np.zeros(n)
    for i in range(n):
        if not ok[i]:
            continue
        d = sorted(math.sqrt(((P[i] - P[j]) ** 2).sum()) for j in range(n) if j != i and ok[j])
        if d:
            out[i] = sum(d[:k]) / len(d[:k])
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    pos = rng.normal(size=(300, 3)) * np.array([1.0, 0.3, 2.0])
    pos[:20] = pos[20:40]  # duplicates: neighbours at distance 0
    np.testing.assert_allclose(oracle.init_point_sizes(pos), _brute(pos), rtol=1e-12, atol=1e-15)


def test_cubic_lattice():
    """Interior points of a cubic lattice of spacing h have six neighbours at h: size h."""
    h = 0.37
    g = np.arange(7) * h
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    s = oracle.init_point_sizes(pos).reshape(7, 7, 7)
    np.testing.assert_allclose(s[1:-1, 1:-1, 1:-1], h, rtol=1e-12)
    # a corner has 3 neighbours at h, then 3 at h sqrt 2: (3 h + h sqrt 2) / 4
    np.testing.assert_allclose(s[0, 0, 0], (3 * h + h * math.sqrt(2)) / 4, rtol=1e-12)


def test_points_on_a_line():
    """Interior points of a line of spacing h: neighbours at h, h, 2h, 2h -> 1.5 h."""
    h = 0.25
    pos = np.stack([np.arange(20) * h, np.zeros(20), np.zeros(20)], 1)
    s = oracle.init_point_sizes(pos)
    np.testing.assert_allclose(s[2:-2], 1.5 * h, rtol=1e-12)
    np.testing.assert_allclose(s[0], (1 + 2 + 3 + 4) * h / 4, rtol=1e-12)


def test_small_and_degenerate_inputs():
    assert oracle.init_point_sizes(np.zeros((1, 3))).tolist() == [0.0]
    s = oracle.init_point_sizes(np.array([[0.0, 0, 0], [3.0, 4.0, 0]]))  # one other point
    np.testing.assert_allclose(s, [5.0, 5.0])
    pos = np.array([[0.0, 0, 0], [1.0, 0, 0], [np.nan, 0, 0], [0, 2.0, 0]])
    s = oracle.init_point_sizes(pos)
    assert s[2] == 0.0
    np.testing.assert_allclose(s[[0, 1, 3]], _brute(pos)[[0, 1, 3]])
