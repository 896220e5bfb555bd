"""Pins of the oracle's coarse-layer inclusion (Sec. 3.6, Implementation Details; reading R24).

With inclusion, the list of pixel (L, j, k) also holds the fragments of every
coarser layer's pixel that contains it, (j >> (L'-L), k >> (L'-L)), each with
its own weight; lists are ordered by (depth, point index, layer).  Pinned by a
pixel-by-pixel definition with hat functions, a closed-form occlusion case,
the all-fine case that reduces to no inclusion, and central differences of
the whole frame for the adjoint.
"""
import math

import numpy as np
import pytest

import oracle

from test_oracle_pins import _cam


def brute_force_coarse(cam, W, H, n_layers, K, pos, sw, alpha, desc, eps=0.25):
    """Each pixel's candidate list built from its definition: its own taps
    (hat functions, Eq. 4-5) and the taps of the coarser pixels above it."""
    cam = np.asarray(cam, np.float64)
    fx, fy, cx, cy = cam[:4]
    R = cam[4:13].reshape(3, 3)
    t = cam[13:16]
    znear = cam[16]
    P = np.asarray(pos, np.float64)
    Xc = P @ R.T + t
    D = desc.shape[1]
    own = {}
    for i in range(P.shape[0]):
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
            for k in range(HL):
                by = max(0.0, 1.0 - abs(y / 2**L - (k + 0.5)))
                for j in range(WL):
                    bx = max(0.0, 1.0 - abs(x / 2**L - (j + 0.5)))
                    if bx * by * iota > 0.0:
                        own.setdefault((L, j, k), []).append((zc, i, L, bx * by * iota))
    off, lw, lh = oracle.pyramid_layout(W, H, n_layers)
    Ptot = int(off[-1])
    pyr = np.zeros((Ptot, D))
    kept = np.full((Ptot, K), -1, np.int64)
    nfrag = np.zeros(Ptot, np.int64)
    tfin = np.ones(Ptot)
    for L in range(n_layers):
        for k in range(int(lh[L])):
            for j in range(int(lw[L])):
                frs = []
                for Lc in range(L, n_layers):
                    frs += own.get((Lc, j >> (Lc - L), k >> (Lc - L)), [])
                p = off[L] + k * lw[L] + j
                frs.sort(key=lambda e: (e[0], e[1], e[2]))
                nfrag[p] = len(frs)
                front = frs[:K]
                gam = [w * float(alpha[i]) for (_, i, _, w) in front]
                T = 1.0
                for m, (_, i, _, _) in enumerate(front):
                    pyr[p] += T * gam[m] * desc[i].astype(np.float64)
                    T *= 1.0 - gam[m]
                    kept[p, m] = i
                tfin[p] = T
    return pyr, kept, nfrag, tfin


def _tiny(seed, n=40, W=21, H=19):
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.5, 0.5, n), rng.uniform(0.6, 2.5, n)], 1)
    sw = np.exp(rng.uniform(math.log(2e-3), math.log(0.6), n))
    alpha = rng.uniform(0.1, 1.0, n)
    desc = rng.uniform(0, 1, (n, 3))
    return (pos.astype(np.float32), sw.astype(np.float32), alpha.astype(np.float32), desc.astype(np.float32),
            _cam(15.0, W, H), W, H)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_coarse_inclusion_brute_force(seed):
    pos, sw, alpha, desc, cam, W, H = _tiny(seed)
    n_layers, K = 4, 4
    fr = oracle.Frame(cam, W, H, n_layers, K, pos, sw, alpha, desc, prec32=False, coarse=True)
    out = fr.render()
    pyr, kept, nfrag, tfin = brute_force_coarse(cam, W, H, n_layers, K, pos, sw, alpha, desc)
    plain = oracle.Frame(cam, W, H, n_layers, K, pos, sw, alpha, desc, prec32=False).render()
    assert (out["n_frag"] > plain["n_frag"]).any(), "coarse fragments must join some fine lists"
    assert (nfrag > K).any(), "the K cap must be exercised"
    np.testing.assert_array_equal(out["n_frag"], nfrag)
    np.testing.assert_array_equal(out["kept"], kept)
    np.testing.assert_allclose(out["pyramid"], pyr, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(out["t_final"], tfin, rtol=1e-12, atol=1e-13)


def test_coarse_inclusion_changes_nothing_without_coarse_fragments():
    """All points below one pixel: every fragment is in layer 0, nothing to include."""
    rng = np.random.default_rng(5)
    n, W, H = 200, 32, 24
    pos = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.4, 0.4, n), rng.uniform(1.0, 2.0, n)], 1)
    sw = np.full(n, 1e-3)
    alpha = rng.uniform(0.1, 1.0, n)
    desc = rng.uniform(0, 1, (n, 4))
    args = (_cam(20.0, W, H), W, H, 4, 8, pos.astype(np.float32), sw.astype(np.float32), alpha.astype(np.float32),
            desc.astype(np.float32))
    a = oracle.Frame(*args, coarse=True).render()
    b = oracle.Frame(*args).render()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_opaque_coarse_point_occludes_the_fine_layers():
    """A point of screen size exactly 4 (layer 2 only, iota = 1) at the centre of
    a layer-2 pixel with alpha = 1 has gamma = 1 there; in front of small
    points it hides them in every finer pixel under that coarse pixel: C is its
    descriptor and the transmittance after it is 0.  Without inclusion the fine
    layers show the small points."""
    W = H = 16
    f, zb, zf = 16.0, 1.0, 3.0
    jc, kc = 1, 2                                  # layer-2 pixel; centre at full-res ((1.5) 4, (2.5) 4)
    xb, yb = (jc + 0.5) * 4, (kc + 0.5) * 4
    big = [(xb - W / 2) * zb / f, (yb - H / 2) * zb / f, zb]
    rng = np.random.default_rng(9)
    small = np.stack([rng.uniform(4.5, 7.5, 30), rng.uniform(8.5, 11.5, 30)], 1)  # under that coarse pixel
    pos = [big] + [[(x - W / 2) * zf / f, (y - H / 2) * zf / f, zf] for x, y in small]
    pos = np.asarray(pos, np.float32)
    sw = np.asarray([4.0 * zb / f] + [0.3 * zf / f] * 30, np.float32)
    alpha = np.asarray([1.0] + [0.8] * 30, np.float32)
    desc = rng.uniform(0, 1, (31, 4)).astype(np.float32)
    off, lw, _ = oracle.pyramid_layout(W, H, 3)
    fr = oracle.Frame(_cam(f, W, H), W, H, 3, 16, pos, sw, alpha, desc, prec32=False, coarse=True)
    out = fr.render()
    plain = oracle.Frame(_cam(f, W, H), W, H, 3, 16, pos, sw, alpha, desc, prec32=False).render()
    covered = 0
    for L in (0, 1):
        d = 2 - L
        for k in range(kc << d, (kc + 1) << d):
            for j in range(jc << d, (jc + 1) << d):
                p = off[L] + k * lw[L] + j
                np.testing.assert_allclose(out["pyramid"][p], desc[0], rtol=0, atol=1e-12)
                assert out["t_final"][p] == 0.0 and out["kept"][p, 0] == 0
                covered += plain["n_frag"][p] > 0
    assert covered > 0, "the small points must reach the covered fine pixels"


def test_coarse_adjoint_matches_frame_differences():
    """Adjoint of a frame with inclusion against central differences of the
    whole frame's loss, in float64, for inputs whose discrete state (taps,
    layers, kept lists) stays the same at +-h."""
    pos, sw, alpha, desc, cam, W, H = _tiny(3, n=30)
    n_layers, K = 4, 6
    G = np.random.default_rng(4).uniform(-1, 1, (int(oracle.pyramid_layout(W, H, n_layers)[0][-1]), 3))

    def frame(p, s, a, d):
        return oracle.Frame(cam, W, H, n_layers, K, p, s, a, d, prec32=False, coarse=True)

    base = frame(pos, sw, alpha, desc)
    g = base.backward(G)
    kept0 = base.render()["kept"]
    checked = 0
    for i in range(len(pos)):
        for what, h in (("pos0", 1e-4), ("pos1", 1e-4), ("pos2", 1e-4), ("sw", 1e-6), ("alpha", 1e-4)):
            vals, used = [], []
            for sgn in (1, -1):
                p, s, a = pos.copy(), sw.copy(), alpha.copy()  # float32, as the frame stores them
                if what.startswith("pos"):
                    p[i, int(what[3])] = np.float32(p[i, int(what[3])] + sgn * h)
                    used.append(float(p[i, int(what[3])]))
                elif what == "sw":
                    s[i] = np.float32(s[i] + sgn * h)
                    used.append(float(s[i]))
                else:
                    a[i] = np.float32(a[i] + sgn * h)
                    used.append(float(a[i]))
                out = frame(p, s, a, desc).render()
                if not np.array_equal(out["kept"], kept0):
                    vals = None
                    break
                vals.append(float((out["pyramid"] * G).sum()))
            if vals is None:
                continue
            fd = (vals[0] - vals[1]) / (used[0] - used[1])  # the float32 step actually taken
            ad = {"pos0": g["pos"][i, 0], "pos1": g["pos"][i, 1], "pos2": g["pos"][i, 2], "sw": g["size_w"][i],
                  "alpha": g["opacity"][i]}[what]
            assert abs(ad - fd) <= 2e-4 * max(1.0, abs(fd)), (i, what, ad, fd)
            checked += 1
    assert checked > 60


def test_point_selection_covers_the_coarse_lists():
    """A frame over selected points holds every list their fragments join
    (with inclusion, also the finer pixels below a coarse fragment), so their
    gradients equal those of the whole frame."""
    pos, sw, alpha, desc, cam, W, H = _tiny(6, n=60, W=40, H=36)
    n_layers, K = 5, 6
    G = np.random.default_rng(7).uniform(-1, 1, (int(oracle.pyramid_layout(W, H, n_layers)[0][-1]), 3))
    full = oracle.Frame(cam, W, H, n_layers, K, pos, sw, alpha, desc, prec32=False, coarse=True)
    g_full = full.backward(G)
    pts = np.arange(0, 60, 7)
    sub = oracle.Frame(cam, W, H, n_layers, K, pos, sw, alpha, desc, prec32=False, coarse=True, points=pts)
    rows = sub.pixels()
    g_sub = sub.backward(G[rows])
    plain_rows = oracle.Frame(cam, W, H, n_layers, K, pos, sw, alpha, desc, prec32=False, points=pts).pixels()
    assert len(rows) > len(plain_rows), "coarse fragments must add finer pixels"
    for k in ("pos", "size_w", "opacity", "desc"):
        np.testing.assert_allclose(g_sub[k][pts], g_full[k][pts], rtol=1e-12, atol=1e-14)
