"""Shared helpers of the GPU parity tests: run the CUDA path, run the oracle, compare."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2401_06003_gb300 import Renderer

# Tolerances for float32 results against the float64 oracle.  A pixel value
# is a chain of at most K = 16 float32 blend steps (relative rounding ~1e-6),
# so 1e-5 leaves headroom; bfloat16 descriptors are rounded to 8 significant
# bits (relative 2^-9), so a pyramid made from them is held to 1e-2 against
# the float32 originals; gradients are sums of float atomics in arbitrary
# order, held to 1e-3.  Gradients with bfloat16 descriptors are compared with
# the oracle run on the same bfloat16-rounded values.
PYR_RTOL = 1e-5      # pyramid values and T_final, float32 descriptors
BF16_RTOL = 1e-2     # pyramid from bfloat16 descriptors vs the oracle on the float32 originals
GRAD_RTOL = 1e-3     # gradients
FLOOR = 1e-3         # relative floor: |g - o| <= rtol * (|o| + FLOOR * max|o|)


def device():
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need CUDA")
    return torch.device("cuda", 0)


def to_dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=device(), dtype=dtype).contiguous()


def gpu_frame(scene, view=0, K=None, mode="store", tile=(16, 8), desc_dtype=torch.float32, desc=None,
              capacity=0, pos=None, expect_flags=0, coarse=False, camera=None):
    """Render one view on the GPU with every optional output; numpy results.

    The device status flags must equal ``expect_flags`` (None: not checked)."""
    cam = scene.cameras[view] if camera is None else camera
    K = K or scene.K
    d = scene.desc if desc is None else desc
    r = Renderer(cam, scene.n_layers, K=K, D=d.shape[1], desc_dtype=desc_dtype, mode=mode, tile=tile,
                 device=device(), coarse=coarse)
    t_pos = to_dev(scene.pos if pos is None else pos)
    t_sw = to_dev(scene.size_w)
    t_op = to_dev(scene.opacity)
    t_desc = to_dev(d, desc_dtype)
    ws = r.new_workspace(scene.n, capacity)
    fr = r.render(t_pos, t_sw, t_op, t_desc, store_lists=True, stats=True, ws=ws)
    flags = r.status(ws)
    out = dict(
        records=fr.records.cpu().numpy(),
        pyramid=fr.pyramid.cpu().numpy(),
        kept=fr.kept.cpu().numpy(),
        n_kept=fr.n_kept.cpu().numpy().astype(np.int32),
        t_final=fr.t_final.cpu().numpy(),
        n_frag=fr.n_frag.cpu().numpy(),
        flags=flags,
    )
    if expect_flags is not None:
        assert flags == expect_flags, f"device status flags {flags:#x}, expected {expect_flags:#x}"
    return r, fr, (t_pos, t_sw, t_op, t_desc), out


def assert_close_scaled(got, ref, rtol, floor=FLOOR, name="", segments=None):
    """|got - ref| <= rtol * (|ref| + floor * max|ref|), the max taken per segment."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape, (name, got.shape, ref.shape)
    segs = segments or [(0, ref.shape[0])]
    for a, b in segs:
        g, o = got[a:b], ref[a:b]
        if o.size == 0:
            continue
        scale = np.abs(o).max()
        err = np.abs(g - o)
        lim = rtol * (np.abs(o) + floor * scale) + 1e-30
        bad = err > lim
        if bad.any():
            idx = np.argwhere(bad)[:5]
            raise AssertionError(f"{name}: {bad.sum()} of {o.size} outside tolerance; worst "
                                 f"{(err / lim).max():.3g}x; first {idx.tolist()} got {g[bad][:5]} want {o[bad][:5]}")


def compare_forward(out, ofr_out, layer_offsets, rtol=PYR_RTOL, rows=None, name=""):
    """Element-wise: kept ids, n_kept and n_frag exact; pyramid and T_final within rtol."""
    sel = slice(None) if rows is None else rows
    kept = out["kept"][sel].astype(np.int64)  # uint32 ids read as int32: 0xFFFFFFFF is -1
    np.testing.assert_array_equal(out["n_frag"][sel].astype(np.int64), ofr_out["n_frag"], err_msg=f"{name} n_frag")
    np.testing.assert_array_equal(out["n_kept"][sel], ofr_out["n_kept"], err_msg=f"{name} n_kept")
    np.testing.assert_array_equal(kept, ofr_out["kept"].astype(np.int64), err_msg=f"{name} kept lists")
    segs = None
    if rows is None:
        segs = [(layer_offsets[L], layer_offsets[L + 1]) for L in range(len(layer_offsets) - 1)]
    assert_close_scaled(out["pyramid"][sel], ofr_out["pyramid"], rtol, name=f"{name} pyramid", segments=segs)
    np.testing.assert_allclose(out["t_final"][sel], ofr_out["t_final"], rtol=rtol, atol=1e-6,
                               err_msg=f"{name} T_final")


def compare_records(gpu_rec, ofr):
    """Projected records are bit-identical to the oracle's float32 projection."""
    xyzs, vis = ofr.records()
    np.testing.assert_array_equal(gpu_rec.astype(np.float64), xyzs)
    assert ((gpu_rec[:, 2] > 0) == (vis == 1)).all()


def oracle_grads_flat(g):
    return dict(pos=g["pos"], size_w=g["size_w"], opacity=g["opacity"], desc=g["desc"])


def compare_grads(gpu, ref, rtol=GRAD_RTOL, name=""):
    for k in ("pos", "size_w", "opacity", "desc"):
        assert_close_scaled(gpu[k].reshape(ref[k].shape[0], -1), ref[k].reshape(ref[k].shape[0], -1), rtol,
                            name=f"{name} grad_{k}")
