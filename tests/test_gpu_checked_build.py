"""The checking build (libtrips_debug.so, TP_DEBUG): every list, pyramid,
workspace and shared-memory index the kernels compute is tested before use,
and an out-of-range one would set TP_FLAG_BOUNDS.  Frames of every kind run
through it must raise no flag and give the release build's outputs."""
import numpy as np
import pytest
import torch

from gpu_helpers import assert_close_scaled, device, to_dev
from paper_2401_06003_gb300 import BatchRenderer, Renderer, _lib, scenes
from paper_2401_06003_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    return _lib.load(build(debug=True))


def _frame(r, sc, desc_dtype, store):
    pos, sw, op = to_dev(sc.pos), to_dev(sc.size_w), to_dev(sc.opacity)
    desc = to_dev(sc.desc, desc_dtype)
    fr = r.render(pos, sw, op, desc, store_lists=store, stats=True)
    G = to_dev(np.random.default_rng(3).uniform(-1, 1, (r.P, sc.D)).astype(np.float32))
    grads = r.splat_backward(fr.records, op, desc, G, fr.workspace, fr.kept if store else None,
                             fr.n_kept if store else None)
    flags = r.status(fr.workspace)
    outs = [fr.pyramid, fr.kept, fr.n_kept, fr.t_final, fr.n_frag, fr.records]
    return flags, [t.cpu() for t in outs], [t.cpu().numpy() for t in grads]


CASES = [
    dict(scene="cube", tile=(16, 8), K=16, mode="store", dtype=torch.float32, coarse=False),
    dict(scene="cube", tile=(13, 7), K=4, mode="recompute", dtype=torch.float32, coarse=False),
    dict(scene="cube", tile=(32, 4), K=32, mode="recompute", dtype=torch.bfloat16, coarse=False),
    dict(scene="ragged", tile=(16, 8), K=8, mode="recompute", dtype=torch.float32, coarse=True),
    dict(scene="cube", tile=(8, 8), K=16, mode="recompute", dtype=torch.float32, coarse=True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['scene']}-{c['tile']}-K{c['K']}-{c['mode']}"
                         f"{'-coarse' if c['coarse'] else ''}")
def test_checked_build_flags_nothing(dbg, case):
    if case["scene"] == "cube":
        sc = scenes.make_config("cube20k_256")
    else:
        sc = scenes.scene_uniform_cube(n=12_000, seed=11, n_layers=7, K=case["K"])
        sc.cameras = [scenes.camera_at((0.3, 0.2, -2.6), (0.0, 0.0, 0.0), 257, 131)]
    outs = []
    for lib in (None, dbg):
        r = Renderer(sc.camera, sc.n_layers, K=case["K"], D=sc.D, desc_dtype=case["dtype"], mode=case["mode"],
                     tile=case["tile"], device=device(), coarse=case["coarse"])
        if lib is not None:
            r.lib = lib
        flags, o, g = _frame(r, sc, case["dtype"], case["mode"] == "store")
        assert flags == 0, f"device status flags {flags:#x}"
        outs.append((o, g))
    (o0, g0), (o1, g1) = outs
    for a, b in zip(o0, o1):
        assert torch.equal(a, b)
    for a, b, name in zip(g0, g1, ("pos", "size_w", "opacity", "desc")):  # only the atomics' order differs
        assert_close_scaled(b.reshape(sc.n, -1), a.reshape(sc.n, -1), 1e-4, name=f"checked grad_{name}")


def test_checked_build_batch_with_cameras(dbg):
    sc = scenes.scene_uniform_cube(n=6000, seed=3, res=64)
    cams = [scenes.camera_at((0.0, 0.3, -3.0), (0.0, 0.0, 0.0), 96, 64),
            scenes.camera_at((2.0, 0.5, -2.5), (0.0, 0.0, 0.0), 130, 70)]
    br = BatchRenderer(cams, 4, K=8, D=4, tiles=[(16, 8), (8, 8)], device=device(), coarse=True)
    br.lib = dbg
    pos, sw, op, desc = to_dev(sc.pos), to_dev(sc.size_w), to_dev(sc.opacity), to_dev(sc.desc)
    fb = br.render(pos, sw, op, desc, stats=True)
    G = to_dev(np.random.default_rng(4).uniform(-1, 1, (br.P, 4)).astype(np.float32))
    br.splat_backward_cameras(pos, fb.records, op, desc, G, fb.workspace)
    assert br.status(fb.workspace) == 0
