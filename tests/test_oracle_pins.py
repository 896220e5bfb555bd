"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's own formulas: they use values
derived by hand from the paper's equations (tests/golden), closed forms,
invariants, a brute-force evaluation written in a different form (a
bilinear hat function over every pixel instead of floor-based tap
selection), and central finite differences for the adjoint.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle


def _cam(f, W, H, R=None, t=(0.0, 0.0, 0.0), znear=0.01):
    R = np.eye(3) if R is None else np.asarray(R)
    return np.concatenate([[f, f, W / 2.0, H / 2.0], R.reshape(9), np.asarray(t, float), [znear]]).astype(np.float32)


def _frame_from_example(ex, prec32):
    pts = ex["points"]
    pos = np.array([p["pos"] for p in pts], np.float32)
    sw = np.array([p["size_w"] for p in pts], np.float32)
    op = np.array([p["opacity"] for p in pts], np.float32)
    desc = np.array([p["desc"] for p in pts], np.float32)
    return oracle.Frame(np.array(ex["camera"], np.float32), ex["width"], ex["height"], ex["n_layers"], ex["K"],
                        pos, sw, op, desc, prec32=prec32)


# --------------------------------------------------------------------------
# Hand-derived worked examples (Eq. 2-7)
# --------------------------------------------------------------------------

def _examples(golden_dir):
    with open(os.path.join(golden_dir, "hand_examples.json")) as fh:
        return json.load(fh)["examples"]


@pytest.mark.parametrize("prec32", [True, False])
def test_hand_examples(golden_dir, prec32):
    for ex in _examples(golden_dir):
        fr = _frame_from_example(ex, prec32)
        xyzs, vis = fr.records()
        if "screen" in ex:
            np.testing.assert_array_equal(xyzs, np.array(ex["screen"]), err_msg=ex["name"])
            assert vis.all()
        if "fragments" in ex:
            pix, z, idx, w = fr.fragments()
            got = sorted(zip(pix.tolist(), idx.tolist(), w.tolist()))
            want = sorted((f["pixel"], f["point"], f["weight"]) for f in ex["fragments"])
            assert got == want, ex["name"]
        out = fr.render()
        for px in ex["pixels"]:
            np.testing.assert_allclose(out["pyramid"][px["pixel"]], px["C"], rtol=0, atol=1e-15, err_msg=ex["name"])
            assert out["t_final"][px["pixel"]] == pytest.approx(px["T_final"], abs=1e-15)
            if "kept" in px:
                nk = out["n_kept"][px["pixel"]]
                assert out["kept"][px["pixel"], :nk].tolist() == px["kept"], ex["name"]


def test_layout_ceil():
    off, w, h = oracle.pyramid_layout(1920, 1080, 8)
    assert w.tolist() == [1920, 960, 480, 240, 120, 60, 30, 15]
    assert h.tolist() == [1080, 540, 270, 135, 68, 34, 17, 9]
    assert off[-1] == 2_764_845
    off, w, h = oracle.pyramid_layout(257, 131, 3)
    assert w.tolist() == [257, 129, 65] and h.tolist() == [131, 66, 33]


# --------------------------------------------------------------------------
# Projection closed forms (Sec. 3.1, Eq. 2)
# --------------------------------------------------------------------------

def test_optical_axis_and_size():
    W, H, f = 64, 48, 50.0
    z = np.array([0.5, 1.0, 2.0, 7.0], np.float32)
    pos = np.stack([np.zeros(4), np.zeros(4), z], 1).astype(np.float32)
    sw = np.array([0.01, 0.02, 0.04, 0.5], np.float32)
    fr = oracle.Frame(_cam(f, W, H), W, H, 4, 16, pos, sw, np.ones(4, np.float32), np.ones((4, 4), np.float32),
                      prec32=False)
    xyzs, vis = fr.records()
    assert vis.all()
    np.testing.assert_allclose(xyzs[:, 0], W / 2)
    np.testing.assert_allclose(xyzs[:, 1], H / 2)
    np.testing.assert_allclose(xyzs[:, 2], z)
    np.testing.assert_allclose(xyzs[:, 3], f * sw.astype(np.float64) / z, rtol=1e-15)


def _random_rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_rigid_motion_invariance():
    """Moving the world and the camera by the same rigid motion leaves the image unchanged."""
    rng = np.random.default_rng(3)
    n, W, H = 200, 40, 30
    pos = rng.uniform(-1, 1, (n, 3))
    sw = rng.uniform(0.005, 0.2, n)
    op = rng.uniform(0.1, 1, n).astype(np.float32)
    desc = rng.uniform(0, 1, (n, 4)).astype(np.float32)
    t = np.array([0.0, 0.0, 3.0])
    base = oracle.Frame(_cam(30.0, W, H, t=t), W, H, 4, 8, pos.astype(np.float32), sw.astype(np.float32), op, desc,
                        prec32=False)
    Q = _random_rotation(rng)
    d = rng.uniform(-1, 1, 3)
    # world' = Q world + d; camera R' = Q^T (so R' Q = I), t' = t - R' d.
    Rp = Q.T
    tp = t - Rp @ d
    posp = pos @ Q.T + d
    # float32 storage of the moved inputs changes them slightly: compare with tolerance.
    moved = oracle.Frame(_cam(30.0, W, H, R=Rp, t=tp), W, H, 4, 8, posp.astype(np.float32),
                         sw.astype(np.float32), op, desc, prec32=False)
    a, _ = base.records()
    b, _ = moved.records()
    np.testing.assert_allclose(a, b, rtol=2e-5, atol=2e-4)


# --------------------------------------------------------------------------
# Weights: partition of unity and the special cases (Eq. 3-5)
# --------------------------------------------------------------------------

def _interior_points(rng, n, s_lo, s_hi, W=256, H=256, f=256.0, z=2.0, n_layers=5):
    """Points whose taps are all inside the image, with screen sizes in [s_lo, s_hi)."""
    margin = 2.0 ** n_layers
    x = rng.uniform(margin, W - margin, n)
    y = rng.uniform(margin, H - margin, n)
    s = rng.uniform(s_lo, s_hi, n)
    pos = np.stack([(x - W / 2) * z / f, (y - H / 2) * z / f, np.full(n, z)], 1)
    return pos.astype(np.float32), (s * z / f).astype(np.float32)


@pytest.mark.parametrize("prec32", [True, False])
@pytest.mark.parametrize("s_lo,s_hi", [(0.01, 0.999), (1.0, 16.0), (16.0, 200.0)])
def test_partition_of_unity(prec32, s_lo, s_hi):
    rng = np.random.default_rng(11)
    n, n_layers, eps = 300, 5, 0.25
    pos, sw = _interior_points(rng, n, s_lo, s_hi, n_layers=n_layers)
    fr = oracle.Frame(_cam(256.0, 256, 256), 256, 256, n_layers, 16, pos, sw, np.ones(n, np.float32),
                      np.ones((n, 4), np.float32), prec32=prec32)
    pix, z, idx, w = fr.fragments()
    total = np.bincount(idx, weights=w, minlength=n)
    xyzs, _ = fr.records()
    s = xyzs[:, 3]
    expect = np.where(s < 1.0, eps + (1 - eps) * s, 1.0)
    np.testing.assert_allclose(total, expect, rtol=1e-12, atol=1e-12)
    counts = np.bincount(idx, minlength=n)
    assert counts.max() <= (4 if s_hi <= 1.0 else 8)
    if s_lo >= 16.0:  # beyond the coarsest layer (2^(5-1) = 16): one layer, at most 4 taps
        assert counts.max() <= 4


def test_integer_layer_pixel_centre_single_tap():
    """A point at a pixel centre of layer L with s = 2^L writes one tap of weight 1."""
    W = H = 128
    f, z = 128.0, 2.0
    for L in range(0, 4):
        for (j, k) in [(0, 0), (3, 5), (7, 2)]:
            x, y = (j + 0.5) * 2**L, (k + 0.5) * 2**L
            pos = np.array([[(x - W / 2) * z / f, (y - H / 2) * z / f, z]], np.float32)
            sw = np.array([2.0**L * z / f], np.float32)
            for prec32 in (True, False):
                fr = oracle.Frame(_cam(f, W, H), W, H, 5, 16, pos, sw, np.ones(1, np.float32),
                                  np.ones((1, 4), np.float32), prec32=prec32)
                pix, _, _, w = fr.fragments()
                off, lw, _ = oracle.pyramid_layout(W, H, 5)
                assert pix.tolist() == [off[L] + k * lw[L] + j]
                assert w.tolist() == [1.0]


def test_layer_weights_linear_in_size():
    """Between 2^L and 2^(L+1) the upper-layer share grows linearly with s (Eq. 5)."""
    W = H = 256
    f, z = 256.0, 2.0
    s = np.array([2.0, 2.5, 3.0, 3.5, 3.999], np.float64)
    x = y = 128.0 + 4.0  # pixel centre at layers 0-2
    pos = np.tile([[(x - W / 2) * z / f, (y - H / 2) * z / f, z]], (s.size, 1)).astype(np.float32)
    sw = (s * z / f).astype(np.float32)
    fr = oracle.Frame(_cam(f, W, H), W, H, 5, 16, pos, sw, np.ones(s.size, np.float32),
                      np.ones((s.size, 4), np.float32), prec32=False)
    pix, _, idx, w = fr.fragments()
    off, _, _ = oracle.pyramid_layout(W, H, 5)
    upper = np.zeros(s.size)
    for p, i, wt in zip(pix, idx, w):
        if p >= off[2]:
            upper[i] += wt
    np.testing.assert_allclose(upper, (s - 2.0) / 2.0, atol=1e-12)


# --------------------------------------------------------------------------
# Brute force on tiny inputs: hat functions over every pixel, full sort
# --------------------------------------------------------------------------

def brute_force(cam, W, H, n_layers, K, pos, sw, alpha, desc, eps=0.25):
    """The paper's definition evaluated pixel by pixel in float64.

    For every layer L, every pixel (j, k) of it and every point, beta is the
    product of the hat functions max(0, 1 - |x/2^L - (j+0.5)|) along x and y
    (Eq. 4), iota comes from Eq. 5 with s_i = 2^L for the point's two layers.
    Every pixel keeps its K nearest fragments by (depth, index) and blends
    them with explicit products T_m = prod_{i<m}(1 - alpha_i) (Eq. 6-7).
    """
    cam = np.asarray(cam, np.float64)
    fx, fy, cx, cy = cam[:4]
    R = cam[4:13].reshape(3, 3)
    t = cam[13:16]
    znear = cam[16]
    P = np.asarray(pos, np.float64)
    Xc = P @ R.T + t
    n = P.shape[0]
    D = desc.shape[1]
    lists = {}
    for i in range(n):
        zc = Xc[i, 2]
        if not zc > znear:
            continue
        x = fx * Xc[i, 0] / zc + cx
        y = fy * Xc[i, 1] / zc + cy
        s = fx * float(sw[i]) / zc
        if s < 1.0:
            layers = [(0, eps + (1 - eps) * s)]
        else:
            lo, hi = math.floor(math.log2(s)), math.ceil(math.log2(s))
            if lo >= n_layers - 1:
                layers = [(n_layers - 1, 1.0)]
            elif lo == hi:
                layers = [(lo, 1.0)]
            else:
                layers = [(L, 1.0 - abs(s - 2.0**L) / (2.0**hi - 2.0**lo)) for L in (lo, hi)]
        for L, iota in layers:
            WL, HL = -(-W // 2**L), -(-H // 2**L)
            xl, yl = x / 2**L, y / 2**L
            for k in range(HL):
                by = max(0.0, 1.0 - abs(yl - (k + 0.5)))
                if by == 0.0:
                    continue
                for j in range(WL):
                    bx = max(0.0, 1.0 - abs(xl - (j + 0.5)))
                    if bx == 0.0 or iota == 0.0:
                        continue
                    lists.setdefault((L, j, k), []).append((zc, i, bx * by * iota))
    off, lw, _ = oracle.pyramid_layout(W, H, n_layers)
    Ptot = int(off[-1])
    pyr = np.zeros((Ptot, D))
    kept = np.full((Ptot, K), -1, np.int64)
    nfrag = np.zeros(Ptot, np.int64)
    tfin = np.ones(Ptot)
    for (L, j, k), frs in lists.items():
        p = off[L] + k * lw[L] + j
        frs.sort(key=lambda e: (e[0], e[1]))
        nfrag[p] = len(frs)
        front = frs[:K]
        gam = [w * float(alpha[i]) for (_, i, w) in front]
        for m, (_, i, _) in enumerate(front):
            Tm = 1.0
            for q in range(m):
                Tm *= 1.0 - gam[q]
            pyr[p] += Tm * gam[m] * desc[i].astype(np.float64)
            kept[p, m] = i
        tfin[p] = float(np.prod([1.0 - g for g in gam])) if gam else 1.0
    return pyr, kept, nfrag, tfin


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    n, W, H, n_layers, K = 48, 23, 17, 4, 3
    pos = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.5, 0.5, n), rng.uniform(0.6, 2.5, n)], 1)
    pos = pos.astype(np.float32)
    # sizes spread over s < 1, two-layer sizes and beyond the coarsest layer
    sw = np.exp(rng.uniform(math.log(2e-3), math.log(0.6), n)).astype(np.float32)
    alpha = rng.uniform(0.1, 1.0, n).astype(np.float32)
    desc = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    cam = _cam(15.0, W, H)
    fr = oracle.Frame(cam, W, H, n_layers, K, pos, sw, alpha, desc, prec32=False)
    out = fr.render()
    pyr, kept, nfrag, tfin = brute_force(cam, W, H, n_layers, K, pos, sw, alpha, desc)
    assert (nfrag > K).any(), "the K cap must be exercised"
    np.testing.assert_array_equal(out["n_frag"], nfrag)
    np.testing.assert_array_equal(out["kept"], kept)
    np.testing.assert_array_equal(out["n_kept"], np.minimum(nfrag, K))
    np.testing.assert_allclose(out["pyramid"], pyr, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(out["t_final"], tfin, rtol=1e-12, atol=1e-13)


def test_ties_broken_by_index_and_cap():
    """Equal depths are ordered by point index; the first K are kept."""
    W = H = 32
    f, z = 32.0, 2.0
    n, K = 20, 5
    x = y = 16.5  # pixel centre of (16, 16) at layer 0
    pos = np.tile([[(x - W / 2) * z / f, (y - H / 2) * z / f, z]], (n, 1)).astype(np.float32)
    sw = np.full(n, 0.5 * z / f, np.float32)  # s = 0.5: layer 0, one tap
    perm = np.random.default_rng(5).permutation(n)
    pos, sw = pos[perm], sw[perm]
    fr = oracle.Frame(_cam(f, W, H), W, H, 3, K, pos, sw, np.full(n, 0.5, np.float32),
                      np.ones((n, 2), np.float32), prec32=True)
    out = fr.render()
    p = 16 * W + 16
    assert out["n_frag"][p] == n
    assert out["kept"][p].tolist() == list(range(K))


def test_empty_culled_and_bad_inputs():
    W = H = 16
    cam = _cam(16.0, W, H, t=(0.0, 0.0, 0.0))
    fr = oracle.Frame(cam, W, H, 2, 4, np.zeros((0, 3), np.float32), np.zeros(0, np.float32),
                      np.zeros(0, np.float32), np.zeros((0, 4), np.float32))
    out = fr.render()
    assert fr.n_frag == 0 and out["pyramid"].sum() == 0 and (out["t_final"] == 1).all()
    pos = np.array([[0, 0, -1.0], [0, 0, 0.005], [np.nan, 0, 1.0], [0, 0, 1.0], [0, 0, 1.0]], np.float32)
    sw = np.array([0.1, 0.1, 0.1, -0.1, np.inf], np.float32)
    fr = oracle.Frame(cam, W, H, 2, 4, pos, sw, np.ones(5, np.float32), np.ones((5, 4), np.float32))
    _, vis = fr.records()
    assert vis.tolist() == [0, 0, 0, 0, 0]
    assert fr.n_bad == 3 and fr.n_frag == 0


def test_prec32_close_to_prec64():
    """The float32 projection stage differs from float64 by rounding only."""
    rng = np.random.default_rng(7)
    n, W, H = 5000, 320, 240
    pos = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(1, 4, n)], 1).astype(np.float32)
    sw = rng.uniform(0.001, 0.05, n).astype(np.float32)
    args = (_cam(240.0, W, H), W, H, 5, 16, pos, sw, np.ones(n, np.float32), np.ones((n, 4), np.float32))
    a, va = oracle.Frame(*args, prec32=True).records()
    b, vb = oracle.Frame(*args, prec32=False).records()
    assert (va == vb).all()
    np.testing.assert_allclose(a[:, :2], b[:, :2], atol=1e-3)
    np.testing.assert_allclose(a[:, 2:], b[:, 2:], rtol=1e-6)


# --------------------------------------------------------------------------
# Adjoint against central finite differences (float64 frames)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_adjoint_matches_finite_differences(seed):
    rng = np.random.default_rng(100 + seed)
    n, W, H, n_layers, K, D = 60, 40, 28, 4, 4, 3
    pos = np.stack([rng.uniform(-0.7, 0.7, n), rng.uniform(-0.5, 0.5, n), rng.uniform(1.0, 3.0, n)], 1)
    pos = pos.astype(np.float32)
    sw = np.exp(rng.uniform(math.log(3e-3), math.log(0.5), n)).astype(np.float32)
    alpha = rng.uniform(0.1, 0.95, n).astype(np.float32)
    desc = rng.uniform(-1, 1, (n, D)).astype(np.float32)
    fr = oracle.Frame(_cam(25.0, W, H), W, H, n_layers, K, pos, sw, alpha, desc, prec32=False)
    G = rng.uniform(-1, 1, (fr.n_pix, D))
    g = fr.backward(G)
    fd, valid = fr.finite_differences(G, np.arange(n))
    ad = np.concatenate([g["pos"], g["size_w"][:, None], g["opacity"][:, None], g["desc"]], 1)
    assert valid.mean() > 0.9
    scale = np.abs(fd[valid]).max()
    err = np.abs(ad - fd)[valid]
    assert err.max() <= 1e-6 * scale + 1e-6 * np.abs(fd[valid]).max(), err.max()
    # points with no fragment have zero gradient
    _, vis = fr.records()
    assert np.all(ad[vis == 0] == 0)


def test_float32_frame_adjoint_matches_anchored_differences():
    """In a float32 frame, the adjoint equals float64 differences taken around
    the frame's own float32 screen-space state."""
    rng = np.random.default_rng(7)
    n, W, H, n_layers, K, D = 80, 640, 360, 6, 4, 3
    pos = np.stack([rng.uniform(-0.9, 0.9, n), rng.uniform(-0.5, 0.5, n), rng.uniform(1.0, 3.0, n)], 1)
    pos = pos.astype(np.float32)
    sw = np.exp(rng.uniform(math.log(1e-3), math.log(0.05), n)).astype(np.float32)
    alpha = rng.uniform(0.1, 0.95, n).astype(np.float32)
    desc = rng.uniform(-1, 1, (n, D)).astype(np.float32)
    fr = oracle.Frame(_cam(360.0, W, H), W, H, n_layers, K, pos, sw, alpha, desc, prec32=True)
    G = rng.uniform(-1, 1, (fr.n_pix, D))
    g = fr.backward(G)
    fd, valid = fr.finite_differences(G, np.arange(n))
    ad = np.concatenate([g["pos"], g["size_w"][:, None], g["opacity"][:, None], g["desc"]], 1)
    assert valid.mean() > 0.9
    err = np.abs(ad - fd)[valid]
    assert err.max() <= 1e-6 * np.abs(fd[valid]).max(), err.max()


# --------------------------------------------------------------------------
# Camera adjoint against central finite differences of the camera
# --------------------------------------------------------------------------

def _rotation(ax, ay, az):
    cx, sx, cy, sy, cz, sz = math.cos(ax), math.sin(ax), math.cos(ay), math.sin(ay), math.cos(az), math.sin(az)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_camera_adjoint_matches_camera_differences(seed):
    """dL/d(fx, fy, cx, cy, R, t) against central differences of the whole
    float64 frame in each camera parameter.  The perturbed parameters are
    float32 values; the difference quotient divides by their actual spacing.
    A parameter whose perturbation changes any fragment list (a tap, a layer
    or an order) is skipped: there the frame is not differentiable."""
    rng = np.random.default_rng(300 + seed)
    n, W, H, n_layers, K, D = 120, 48, 36, 4, 4, 3
    pos = np.stack([rng.uniform(-0.8, 0.8, n), rng.uniform(-0.6, 0.6, n), rng.uniform(-0.8, 0.8, n)], 1)
    pos = pos.astype(np.float32)
    sw = np.exp(rng.uniform(math.log(3e-3), math.log(0.3), n)).astype(np.float32)
    alpha = rng.uniform(0.1, 0.95, n).astype(np.float32)
    desc = rng.uniform(-1, 1, (n, D)).astype(np.float32)
    R = _rotation(*rng.uniform(-0.3, 0.3, 3))
    cam = _cam(40.0, W, H, R=R, t=(0.05, -0.1, 3.0))
    cam[1] = 44.0  # fy != fx
    cam[2], cam[3] = 23.5, 18.25

    def frame(c):
        return oracle.Frame(c, W, H, n_layers, K, pos, sw, alpha, desc, prec32=False)

    fr = frame(cam)
    G = rng.uniform(-1, 1, (fr.n_pix, D))
    g = fr.camera_backward(G)
    pix0, _, idx0, _ = fr.fragments()
    steps = [1e-5 * abs(float(cam[q])) for q in range(4)] + [1e-6] * 12
    fd = np.full(16, np.nan)
    for q in range(16):
        cp, cm = cam.copy(), cam.copy()
        cp[q] = np.float32(float(cam[q]) + steps[q])
        cm[q] = np.float32(float(cam[q]) - steps[q])
        fp, fm = frame(cp), frame(cm)
        same = True
        for f_ in (fp, fm):
            pix, _, idx, _ = f_.fragments()
            same = same and pix.shape == pix0.shape and (pix == pix0).all() and (idx == idx0).all()
        if not same:
            continue
        Lp = float((G * fp.render()["pyramid"]).sum())
        Lm = float((G * fm.render()["pyramid"]).sum())
        fd[q] = (Lp - Lm) / (float(cp[q]) - float(cm[q]))
    ok = ~np.isnan(fd)
    assert ok.sum() >= 12, ok
    for sl in (slice(0, 4), slice(4, 13), slice(13, 16)):  # intrinsics, rotation, translation
        m = ok[sl]
        if not m.any():
            continue
        ref, got = fd[sl][m], g[sl][m]
        scale = np.abs(fd[sl][m]).max()
        assert np.all(np.abs(got - ref) <= 1e-4 * (np.abs(ref) + 1e-3 * scale)), (sl, got, ref)
    assert np.abs(g).max() > 0


def test_camera_adjoint_zero_without_visible_points():
    """Points behind the camera carry no camera gradient."""
    n, W, H = 10, 16, 12
    pos = np.stack([np.zeros(n), np.zeros(n), -np.linspace(1, 2, n)], 1).astype(np.float32)
    fr = oracle.Frame(_cam(10.0, W, H), W, H, 2, 4, pos, np.full(n, 0.1, np.float32), np.full(n, 0.5, np.float32),
                      np.ones((n, 2), np.float32), prec32=False)
    assert np.all(fr.camera_backward(np.ones((fr.n_pix, 2))) == 0)
