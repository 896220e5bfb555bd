"""Batches of views (one launch per stage over several cameras) against
single-view renders and the float64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import GRAD_RTOL, assert_close_scaled, compare_forward, compare_records, device, to_dev
from paper_2401_06003_gb300 import BatchRenderer, Renderer, autotune_batch_tiles, autotune_tiles, scenes

pytestmark = pytest.mark.gpu


def _cams():
    """Three cameras of uneven resolution around the cube scene."""
    c0 = scenes.camera_at((0.0, 0.3, -3.0), (0.0, 0.0, 0.0), 96, 64)
    c1 = scenes.camera_at((2.0, 0.5, -2.5), (0.0, 0.0, 0.0), 130, 70)
    c2 = scenes.camera_at((-2.5, -0.4, -2.0), (0.1, 0.0, 0.0), 64, 64)
    return [c0, c1, c2]


@pytest.fixture(scope="module")
def scene():
    return scenes.scene_uniform_cube(n=6000, seed=3, res=64)


def _inputs(sc):
    return to_dev(sc.pos), to_dev(sc.size_w), to_dev(sc.opacity), to_dev(sc.desc)


def test_batch_matches_single_views_and_oracle(scene):
    cams = _cams()
    tiles = [(16, 8), (8, 8), (16, 16)]
    br = BatchRenderer(cams, 4, K=8, D=4, tiles=tiles, mode="store", device=device())
    pos, sw, op, desc = _inputs(scene)
    fb = br.render(pos, sw, op, desc, stats=True)
    assert br.status(fb.workspace) == 0
    for v, cam in enumerate(cams):
        r = Renderer(cam, 4, K=8, D=4, tile=tiles[v], mode="store", device=device())
        fs = r.render(pos, sw, op, desc, stats=True)
        for name in ("pyramid", "kept", "n_kept", "t_final", "n_frag"):
            a = br.view(getattr(fb, name), v)
            b = getattr(fs, name)
            assert torch.equal(a, b), (v, name)
        assert torch.equal(fb.records[v], fs.records)
        sc = scene.subset(np.arange(scene.n))
        sc.cameras, sc.K = [cam], 8
        ofr = oracle.Frame.from_scene(sc)
        compare_records(fs.records.cpu().numpy(), ofr)
        out = dict(pyramid=fs.pyramid.cpu().numpy(), kept=fs.kept.cpu().numpy(),
                   n_kept=fs.n_kept.cpu().numpy().astype(np.int32), t_final=fs.t_final.cpu().numpy(),
                   n_frag=fs.n_frag.cpu().numpy())
        compare_forward(out, ofr.render(), r.layer_offsets, name=f"view {v}")


@pytest.mark.parametrize("mode", ["recompute", "store"])
def test_batch_backward_is_sum_over_views(scene, mode):
    cams = _cams()
    br = BatchRenderer(cams, 4, K=8, D=4, tiles=[(16, 8), (8, 8), (16, 16)], mode=mode, device=device())
    pos, sw, op, desc = _inputs(scene)
    fb = br.render(pos, sw, op, desc)
    G = np.random.default_rng(5).uniform(-1, 1, (br.P, 4)).astype(np.float32)
    got = [t.cpu().numpy() for t in br.backward(fb, op, desc, to_dev(G))]
    ref = [np.zeros((scene.n, 3)), np.zeros(scene.n), np.zeros(scene.n), np.zeros((scene.n, 4))]
    for v, cam in enumerate(cams):
        sc = scene.subset(np.arange(scene.n))
        sc.cameras, sc.K = [cam], 8
        g = oracle.Frame.from_scene(sc).backward(G[br.view_offsets[v]:br.view_offsets[v + 1]].astype(np.float64))
        for q, k in enumerate(("pos", "size_w", "opacity", "desc")):
            ref[q] += g[k]
    for q, k in enumerate(("pos", "size_w", "opacity", "desc")):
        assert_close_scaled(got[q].reshape(scene.n, -1), ref[q].reshape(scene.n, -1), GRAD_RTOL, name=f"sum {k}")


def test_batch_step_replays_as_one_cuda_graph(scene):
    cams = _cams()
    br = BatchRenderer(cams, 4, K=16, D=4, tiles=[(16, 8), (16, 8), (16, 16)], device=device())
    pos, sw, op, desc = _inputs(scene)
    n = scene.n
    ws = br.new_workspace(n)
    rec = torch.empty((br.n_views, n, 4), device=device())
    pyr = torch.empty((br.P, 4), device=device())
    G = (torch.rand((br.P, 4), device=device()) * 2 - 1).contiguous()
    grads = (torch.empty((n, 3), device=device()), torch.empty(n, device=device()), torch.empty(n, device=device()),
             torch.empty((n, 4), device=device()))

    def step():
        br.project(pos, sw, ws, records=rec)
        br.splat_forward(rec, op, ws)
        br.blend(rec, op, desc, ws, pyramid=pyr)
        br.splat_backward(rec, op, desc, G, ws, grads=grads)

    s = torch.cuda.Stream(device())
    s.wait_stream(torch.cuda.current_stream(device()))
    with torch.cuda.stream(s):
        step()  # eager, on the capture stream, sets kernel attributes
    torch.cuda.current_stream(device()).wait_stream(s)
    torch.cuda.synchronize()
    eager = [pyr.clone()] + [g.clone() for g in grads]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(2):
        pyr.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(pyr, eager[0])
        for a, b in zip(grads, eager[1:]):  # same arithmetic; only the order of the float atomics differs
            assert_close_scaled(a.cpu().numpy().reshape(n, -1), b.cpu().numpy().reshape(n, -1), 1e-4,
                                name="replayed gradients")


def test_autotune_picks_a_working_tile(scene):
    cams = _cams()[:2]
    pos, sw, op, desc = _inputs(scene)
    tiles, timings = autotune_tiles(cams, 4, pos, sw, op, desc, candidates=((16, 8), (8, 8), (32, 32)), iters=2,
                                    device=device())
    assert len(tiles) == 2
    for cam, t in zip(cams, tiles):
        res = (cam.width, cam.height)
        assert t in timings[res] and t != (32, 32)  # the oversized tile is refused, never timed
        assert all(ms > 0 for ms in timings[res].values())


def test_orbit16_full_size_sampled():
    """The 6M-point cloud in 16 orbit views of uneven resolution, one batch:
    sampled pixels of four views against the oracle."""
    sc = scenes.make_config("ground6m_orbit16")
    br = BatchRenderer(sc.cameras, sc.n_layers, K=sc.K, D=sc.D, device=device())
    pos, sw, op, desc = _inputs(sc)
    fb = br.render(pos, sw, op, desc, stats=True)
    assert br.status(fb.workspace) == 0
    rng = np.random.default_rng(61)
    for v in (0, 5, 10, 15):
        lo, hi = br.view_offsets[v], br.view_offsets[v + 1]
        pix = rng.choice(hi - lo, size=5000, replace=False)
        ofr = oracle.Frame.from_scene(sc, view=v, pixels=pix)
        rows = ofr.pixels()
        out = dict(pyramid=br.view(fb.pyramid, v).cpu().numpy(), kept=br.view(fb.kept, v).cpu().numpy(),
                   n_kept=br.view(fb.n_kept, v).cpu().numpy().astype(np.int32),
                   t_final=br.view(fb.t_final, v).cpu().numpy(), n_frag=br.view(fb.n_frag, v).cpu().numpy())
        off, _, _ = oracle.pyramid_layout(sc.cameras[v].width, sc.cameras[v].height, sc.n_layers)
        compare_forward(out, ofr.render(), off.tolist(), rows=rows, name=f"orbit view {v}")


def test_batch_autotune_times_the_batch(scene):
    cams = _cams()
    pos, sw, op, desc = _inputs(scene)
    tiles, timings = autotune_batch_tiles(cams, 4, pos, sw, op, desc, candidates=((16, 8), (8, 8), (32, 32)),
                                          iters=2, device=device())
    assert len(tiles) == len(cams)
    for cam, t in zip(cams, tiles):
        res = (cam.width, cam.height)
        assert t in timings[res] and t != (32, 32)  # the oversized tile is refused, never timed
        assert timings[res][t] == min(timings[res].values())
    # the chosen shapes render the batch exactly as the single views do
    br = BatchRenderer(cams, 4, K=8, D=4, tiles=tiles, mode="store", device=device())
    fb = br.render(pos, sw, op, desc)
    for v, cam in enumerate(cams):
        fs = Renderer(cam, 4, K=8, D=4, tile=tiles[v], mode="store", device=device()).render(pos, sw, op, desc)
        assert torch.equal(br.view(fb.pyramid, v), fs.pyramid)


def test_batch_camera_gradients_per_view(scene):
    """One batch backward returns every view's camera gradient (Sec. 3.5):
    each against the oracle's camera adjoint of that view alone, and the point
    gradients equal those of the plain batch backward."""
    cams = _cams()
    br = BatchRenderer(cams, 4, K=8, D=4, tiles=[(16, 8), (8, 8), (16, 16)], device=device())
    pos, sw, op, desc = _inputs(scene)
    fb = br.render(pos, sw, op, desc)
    G = np.random.default_rng(8).uniform(-1, 1, (br.P, 4)).astype(np.float32)
    grads, gcam = br.splat_backward_cameras(pos, fb.records, op, desc, to_dev(G), fb.workspace)
    plain = br.backward(fb, op, desc, to_dev(G))
    for a, b, name in zip(grads, plain, ("pos", "size_w", "opacity", "desc")):
        # same arithmetic; only the order of the float atomics differs
        assert_close_scaled(a.cpu().numpy(), b.cpu().numpy(), 1e-4, name=f"camera-pass grad_{name}")
    groups = [(0, 4), (4, 13), (13, 16)]
    got = gcam.cpu().numpy()
    assert got.shape == (3, 16)
    for v, cam in enumerate(cams):
        sc = scene.subset(np.arange(scene.n))
        sc.cameras, sc.K = [cam], 8
        ref = oracle.Frame.from_scene(sc).camera_backward(
            G[br.view_offsets[v]:br.view_offsets[v + 1]].astype(np.float64))
        assert_close_scaled(got[v], ref, GRAD_RTOL, name=f"view {v} camera gradient", segments=groups)
