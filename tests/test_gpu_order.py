"""Spatial order of a cloud (tp_spatial_order, tp_permute_rows) and renders of relabeled clouds."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import GRAD_RTOL, PYR_RTOL, assert_close_scaled, compare_forward, device, gpu_frame, to_dev
from paper_2401_06003_gb300 import Renderer, permute_rows, scenes, spatial_order

pytestmark = pytest.mark.gpu


def morton_order_reference(pos):
    """The documented order, written out: float32 cell coordinates in a 1024^3
    grid over the finite points' box, bits interleaved x-lowest, stable sort,
    non-finite points last."""
    pos = np.asarray(pos, np.float32)
    fin = np.isfinite(pos).all(1)
    code = np.full(len(pos), 0xFFFFFFFF, np.uint64)
    if fin.any():
        lo = pos[fin].min(0)
        ext = np.float32((pos[fin].max(0) - lo).max())
        scale = np.float32(1023) / ext if ext > 0 else np.float32(0)
        q = ((pos[fin] - lo).astype(np.float32) * scale).astype(np.float32)
        q = np.clip(q.astype(np.int64), 0, 1023)
        c = np.zeros(fin.sum(), np.uint64)
        for b in range(10):
            for a in range(3):
                c |= ((q[:, a] >> b) & 1).astype(np.uint64) << np.uint64(3 * b + a)
        code[fin] = c
    return np.argsort(code, kind="stable")


@pytest.mark.parametrize("n", [1, 1000, 4097, 200_000])
def test_spatial_order_matches_definition(n):
    rng = np.random.default_rng(n)
    pos = rng.normal(size=(n, 3)).astype(np.float32) * np.float32(3)
    if n > 10:
        pos[rng.choice(n, n // 100 + 1, replace=False)] = pos[:n // 100 + 1]  # duplicate cells and codes
        pos[5, 1] = np.nan
        pos[7, 2] = np.inf
    perm = spatial_order(to_dev(pos)).cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(np.sort(perm), np.arange(n))
    np.testing.assert_array_equal(perm, morton_order_reference(pos))


def test_spatial_order_empty_and_flat():
    assert spatial_order(to_dev(np.zeros((0, 3), np.float32))).numel() == 0
    flat = np.zeros((300, 3), np.float32)  # one position: every code 0, identity order
    np.testing.assert_array_equal(spatial_order(to_dev(flat)).cpu().numpy(), np.arange(300))


@pytest.mark.parametrize("cols,dtype", [(1, torch.float32), (3, torch.float32), (16, torch.bfloat16),
                                        (5, torch.int32)])
def test_permute_rows(cols, dtype):
    n = 5000
    t = torch.arange(n * cols, device=device()).reshape(n, cols).to(dtype)
    perm = torch.randperm(n, device=device()).to(torch.int32)
    got = permute_rows(t.contiguous() if cols > 1 else t.reshape(n).contiguous(), perm)
    want = t[perm.long()] if cols > 1 else t.reshape(n)[perm.long()]
    assert torch.equal(got, want)


def test_relabeled_cloud_renders_the_same():
    """The same frame from a Morton-relabeled cloud: identical pyramid, kept lists
    that map back to the original indices, gradients that permute with the points,
    and oracle parity on the relabeled cloud."""
    sc = scenes.make_config("cube20k_256")
    perm = spatial_order(to_dev(sc.pos)).cpu().numpy().astype(np.int64)
    rel = sc.subset(perm)
    r0, fr0, ins0, out0 = gpu_frame(sc, mode="store")
    r1, fr1, ins1, out1 = gpu_frame(rel, mode="store")
    # the cube has no exactly equal depths within a pixel, so the blend order is the same
    np.testing.assert_array_equal(out1["pyramid"], out0["pyramid"])
    k1 = out1["kept"].astype(np.int64)
    mapped = np.where(k1 >= 0, perm[np.maximum(k1, 0)], -1)
    np.testing.assert_array_equal(mapped, out0["kept"].astype(np.int64))
    ofr = oracle.Frame.from_scene(rel)
    compare_forward(out1, ofr.render(), r1.layer_offsets, name="relabeled cube")
    G = np.random.default_rng(3).uniform(-1, 1, (r0.P, sc.D)).astype(np.float32)
    g0 = [t.cpu().numpy() for t in r0.backward(fr0, ins0[2], ins0[3], to_dev(G))]
    g1 = [t.cpu().numpy() for t in r1.backward(fr1, ins1[2], ins1[3], to_dev(G))]
    for a, b, name in zip(g0, g1, ("pos", "size_w", "opacity", "desc")):
        assert_close_scaled(b, a[perm], GRAD_RTOL, name=f"relabeled grad_{name}")
