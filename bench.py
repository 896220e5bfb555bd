#!/usr/bin/env python3
"""Benchmark: forward + backward trilinear point splatting on GB300.

Workload (default): 6M-point scene-shaped cloud (noisy heightfield ground,
Gaussian clusters, far shell; Pareto sizes) rendered at 1920x1080 into 8
pyramid layers, K = 16, D = 4 float32 descriptors, kept lists recomputed in
the backward pass.  One step = project -> splat -> blend -> backward for one
frame with a fixed upstream gradient.  Inputs are resident in HBM when the
timed region starts; the point inputs alone (216 MB) are larger than L2.

Prints one JSON line (rank 0).  ``--impl reference`` times the float64 CPU
oracle on the host cores instead (a bounded random subset of the same cloud
per step).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/frame & Mpoints/s, 6M pts @1080p; % of HBM roofline"
FALLBACK_HBM_GBS = 6800.0
KERNELS_PER_STEP = 6  # k_project_count, k_tile_totals, k_scan_tiles, k_fill, k_tile_blend, k_tile_backward


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ground6m_1080p")
    ap.add_argument("--mode", choices=["recompute", "store"], default="recompute")
    ap.add_argument("--tile", default="16x8")
    ap.add_argument("--points", type=int, default=0, help="override the workload's point count (profiling)")
    ap.add_argument("--desc-dtype", choices=["auto", "f32", "bf16"], default="auto",
                    help="descriptor storage type (auto: bf16 for the *_bf16 workloads)")
    ap.add_argument("--point-order", choices=["spatial", "generation"], default="spatial",
                    help="spatial: relabel the cloud once along a Morton curve (tp_spatial_order, untimed) before "
                         "timing; generation: the order the generator draws (random within each component)")
    ap.add_argument("--cpu-frames", type=int, default=2, help="full oracle frames timed for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the camera-adjoint, pyramid-merge and point-size timings (profiling the step alone)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--copy-streams", type=int, default=1,
                    help="copy streams the end-to-end upload and download are split over")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the summaries of the batched 16-view and 4K bf16 workloads in the default line")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: every rank renders its own frame)
# ---------------------------------------------------------------------------

def dist_setup(use_cuda):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if use_cuda else "gloo")
    if use_cuda:
        torch.cuda.set_device(local)
    return rank, world, local


def barrier(world, device=None):
    import torch.distributed as dist

    if world > 1:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(x, world, device):
    import torch
    import torch.distributed as dist

    if world == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = max(smax, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------

def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# the source files each profiled kernel is compiled from
KERNEL_FILES = {"k_project_count": ("bin.cu", "common.cuh"), "k_fill": ("bin.cu", "common.cuh"),
                "k_tile_blend": ("blend.cu", "common.cuh"), "k_tile_backward": ("blend.cu", "common.cuh")}


def source_hash(files=None):
    """Hash of the kernel sources' code (comments and whitespace removed)."""
    from paper_2401_06003_gb300.build import source_hash as _hash

    return _hash(files)


def accuracy_report(workload):
    """The committed accuracy report of `workload` (pyramid and gradient errors
    against the float64 oracle, written by the GPU parity test), if it was
    taken from the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", f"accuracy_{workload}.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    from paper_2401_06003_gb300.build import RENDER_PATH_FILES

    if d.get("source_hash") != source_hash(RENDER_PATH_FILES):
        return None
    return d


def ncu_traffic(kernel, workload, points):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken from the current kernel sources on this workload and point
    count; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    k = d.get("kernels", {}).get(kernel)
    if not k or k.get("workload") != workload or k.get("points") != points:
        return None
    if k.get("source_hash") != source_hash(KERNEL_FILES.get(kernel)):
        return None
    return k.get("dram_bytes_per_launch")


def algorithmic_bytes(N, V, F, P, D, b):
    """Per-stage algorithmic bytes of one frame (per launch).

    project  : read x, s_w, alpha (20 N) + write the point record (16 V)
    splat    : write each fragment key once (8 F) + the pixel offsets (8 P)
    blend    : read each key once (8 F) + descriptors (b D V) + write the pyramid (4 D P)
    backward : re-read keys (8 F), records and descriptors ((16 + b D) V),
               read dL/dpyramid (4 D P), write the gradients (4 (5 + D) N)
    The first three sum to the forward total 20N + (16 + bD)V + 16F + 8P + 4DP.
    """
    return {
        "project": 20 * N + 16 * V,
        "splat": 8 * F + 8 * P,
        "blend": 8 * F + b * D * V + 4 * D * P,
        "backward": 8 * F + (16 + b * D) * V + 4 * D * P + 4 * (5 + D) * N,
    }


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

def relabel_cloud(args, step, tensors, stream, dev):
    """With --point-order spatial: time `step` on the cloud as generated, then
    relabel every per-point tensor once along the Morton curve of the cloud
    (tp_spatial_order + tp_permute_rows; outside the timed region) and return
    the relabeled tensors (the same for the caller, in place of `tensors`)."""
    import torch

    from paper_2401_06003_gb300 import permute_rows, spatial_order

    if args.point_order != "spatial":
        return {"kind": "generation", "tensors": tensors}
    step_ms = None
    if args.steps > 0:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            step()
        g1.record(stream)
        torch.cuda.synchronize(dev)
        step_ms = g0.elapsed_time(g1) / args.steps
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    perm = spatial_order(tensors[0])
    out = [permute_rows(t, perm) for t in tensors]
    r1.record(stream)
    torch.cuda.synchronize(dev)
    for dst, src in zip(tensors, out):  # the step closure reads the original tensors: overwrite them
        dst.copy_(src)
    torch.cuda.synchronize(dev)
    return {"kind": "spatial (Morton order, tp_spatial_order, once per cloud, untimed)",
            "relabel_ms": round(r0.elapsed_time(r1), 3),
            "generation_order_ms_per_step": None if step_ms is None else round(step_ms, 4),
            "tensors": tensors}


def run_ours(args):
    import torch

    from paper_2401_06003_gb300 import Renderer, scenes
    from paper_2401_06003_gb300.build import build as build_lib

    build_lib()
    rank, world, local = dist_setup(True)
    dev = torch.device("cuda", local)
    sc = scenes.make_config(args.workload, n=args.points or None)
    tw, th = (int(v) for v in args.tile.split("x"))
    if args.desc_dtype == "auto":
        desc_dtype = torch.bfloat16 if args.workload.endswith("bf16") else torch.float32
    else:
        desc_dtype = torch.bfloat16 if args.desc_dtype == "bf16" else torch.float32
    r = Renderer(sc.camera, sc.n_layers, K=sc.K, D=sc.D, desc_dtype=desc_dtype, mode=args.mode, tile=(tw, th),
                 device=dev)
    N, D, P = sc.n, sc.D, r.P
    b = 2 if desc_dtype == torch.bfloat16 else 4

    pos = torch.from_numpy(sc.pos).to(dev)
    sw = torch.from_numpy(sc.size_w).to(dev)
    op = torch.from_numpy(sc.opacity).to(dev)
    desc = torch.from_numpy(sc.desc).to(dev).to(desc_dtype).contiguous()
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + rank)
    G = (torch.rand((P, D), generator=gen, device=dev) * 2 - 1).contiguous()
    ws = r.new_workspace(N)
    rec = torch.empty((N, 4), dtype=torch.float32, device=dev)
    pyr = torch.empty((P, D), dtype=torch.float32, device=dev)
    grads = (torch.empty((N, 4), device=dev), None, torch.empty((N,), device=dev),  # packed (X, Y, Z, s_w) rows
             torch.empty((N, D), device=dev))
    store = args.mode == "store"
    stream = torch.cuda.current_stream(dev)
    # the gradient buffers are cleared on a second stream while the blend runs
    # (it uses little DRAM bandwidth); the backward waits for the clearing
    zero_stream = torch.cuda.Stream(dev)
    zeroed = torch.cuda.Event()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        r.project(pos, sw, ws, records=rec)
        if ev is not None:
            ev[1].record(stream)
        r.splat_forward(rec, op, ws)
        if ev is not None:
            ev[2].record(stream)
        zero_stream.wait_stream(stream)  # also orders it after the previous step's backward
        r.zero_gradients(grads, stream=zero_stream)
        zeroed.record(zero_stream)
        _, kept, nk, _, _ = r.blend(rec, op, desc, ws, store_lists=store, pyramid=pyr)
        if ev is not None:
            ev[3].record(stream)
        stream.wait_event(zeroed)
        r.splat_backward(rec, op, desc, G, ws, kept if store else None, nk if store else None, grads=grads,
                         grads_zeroed=True)
        if ev is not None:
            ev[4].record(stream)

    order = relabel_cloud(args, step, [pos, sw, op, desc], stream, dev)
    pos, sw, op, desc = order.pop("tensors")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    flags = r.status(ws)
    if flags:
        raise RuntimeError(f"device status flags {flags:#x} after warm-up")

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device()) if not args.no_clocks else None
    barrier(world, dev)
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.start()
        time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(args.steps):
        step(evs[s])
    t1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    clk = clocks.stop() if clocks else None
    elapsed_ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    stage_ms = {name: float(np.mean([evs[s][q].elapsed_time(evs[s][q + 1]) for s in range(args.steps)]))
                for q, name in enumerate(["project", "splat", "blend", "backward"])}

    # counters of the frame (untimed)
    _, kept, nk, tfin, nfrag = r.blend(rec, op, desc, ws, stats=True)
    V = int((rec[:, 2] > 0).sum().item())
    F = int(nfrag.to(torch.int64).sum().item())
    Fk = int(nk.to(torch.int64).sum().item())

    ms_per_step = elapsed_ms / args.steps
    value = N * world / (ms_per_step * 1e-3) / 1e6
    A = algorithmic_bytes(N, V, F, P, D, b)
    peak, peak_kind = measured_hbm_peak()
    dom = max(stage_ms, key=stage_ms.get)
    kname = {"project": "k_project_count", "splat": "k_fill", "blend": "k_tile_blend",
             "backward": "k_tile_backward"}[dom]
    achieved = A[dom] / (stage_ms[dom] * 1e-3) / 1e9
    step_bytes = sum(A.values())
    roofline = {
        "bound": "hbm", "kernel": kname, "stage": dom, "achieved": round(achieved, 1), "peak": peak,
        "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
        "traffic": ncu_traffic(kname, args.workload, N),
        "algorithmic_bytes": int(A[dom]),
        "step": {"achieved": round(step_bytes / (ms_per_step * 1e-3) / 1e9, 1),
                 "frac": round(step_bytes / (ms_per_step * 1e-3) / 1e9 / peak, 4),
                 "algorithmic_bytes": int(step_bytes)},
        "stages": {k: {"ms": round(v, 4), "algorithmic_bytes": int(A[k]),
                       "frac": round(A[k] / (v * 1e-3) / 1e9 / peak, 4)} for k, v in stage_ms.items()},
    }

    # end to end through the public API with host buffers: every step copies
    # its inputs from pinned host memory and its gradients back.  Two buffer
    # sets and two copy streams let step k+1's upload and step k-1's download
    # overlap step k's kernels (the renderer's calls take any stream).
    e2e = None
    if not args.no_e2e:
        # the host copy of the cloud is stored in the same (relabeled) order
        h_in = [t.cpu().pin_memory() for t in (pos, sw, op, desc)]
        d_in = [[pos, sw, op, desc], [torch.empty_like(t) for t in (pos, sw, op, desc)]]
        d_gr = [list(grads), [None if g is None else torch.empty_like(g) for g in grads]]
        h_out = [[torch.empty(g.shape, dtype=torch.float32).pin_memory() for g in grads if g is not None]
                 for _ in range(2)]
        # the step's result read back: the loss <G, pyramid> whose gradient is the
        # upstream gradient G (the point gradients stay on the device, as for an
        # optimizer step); a second figure also downloads every gradient
        d_loss = [torch.empty((), dtype=torch.float32, device=dev) for _ in range(2)]
        h_loss = [torch.empty((), dtype=torch.float32).pin_memory() for _ in range(2)]
        h2d = sum(t.numel() * t.element_size() for t in h_in)
        d2h_grads = sum(t.numel() * t.element_size() for t in h_out[0])
        # each tensor's copy is cut into contiguous pieces, one per copy stream
        # (one copy stream alone does not reach the host link's bandwidth)
        n_cs = max(1, args.copy_streams)
        s_in = [torch.cuda.Stream(dev) for _ in range(n_cs)]
        s_out = [torch.cuda.Stream(dev) for _ in range(n_cs)]
        computed = [torch.cuda.Event() for _ in range(2)]
        downloaded = [[torch.cuda.Event() for _ in range(n_cs)] for _ in range(2)]
        uploaded = [[torch.cuda.Event() for _ in range(n_cs)] for _ in range(2)]

        def pieces(dst, src):
            """(stream index, dst piece, src piece) over the copy streams."""
            a_, b_ = dst.view(-1), src.view(-1)
            n_ = a_.numel()
            step = -(-n_ // n_cs)
            step = -(-step // 1024) * 1024
            return [(j, a_[j * step:min(n_, (j + 1) * step)], b_[j * step:min(n_, (j + 1) * step)])
                    for j in range(n_cs) if j * step < n_]

        def pipeline(steps, download_grads):
            for k in range(steps):
                b = k % 2
                if k >= 2:
                    for s_ in s_in:
                        s_.wait_event(computed[b])    # step k-2 no longer reads these inputs
                    for ev in downloaded[b]:
                        stream.wait_event(ev)          # its results are on the host
                for d_, h_ in zip(d_in[b], h_in):
                    for j, dp, hp in pieces(d_, h_):
                        with torch.cuda.stream(s_in[j]):
                            dp.copy_(hp, non_blocking=True)
                for j, s_ in enumerate(s_in):
                    uploaded[b][j].record(s_)
                    stream.wait_event(uploaded[b][j])
                pb, swb, opb, db = d_in[b]
                r.project(pb, swb, ws, records=rec)
                r.splat_forward(rec, opb, ws)
                _, kept_b, nk_b, _, _ = r.blend(rec, opb, db, ws, store_lists=store, pyramid=pyr)
                torch.dot(pyr.view(-1), G.view(-1), out=d_loss[b])
                r.splat_backward(rec, opb, db, G, ws, kept_b if store else None, nk_b if store else None,
                                 grads=tuple(d_gr[b]))
                computed[b].record(stream)
                for s_ in s_out:
                    s_.wait_event(computed[b])
                with torch.cuda.stream(s_out[0]):
                    h_loss[b].copy_(d_loss[b], non_blocking=True)
                if download_grads:
                    for h_, g_ in zip(h_out[b], [g for g in d_gr[b] if g is not None]):
                        for j, hp, gp in pieces(h_, g_):
                            with torch.cuda.stream(s_out[j]):
                                hp.copy_(gp, non_blocking=True)
                for j, s_ in enumerate(s_out):
                    downloaded[b][j].record(s_)
            for s_ in s_out:
                stream.wait_stream(s_)

        def timed_pipeline(download_grads):
            pipeline(min(args.warmup, 3), download_grads)
            torch.cuda.synchronize(dev)
            barrier(world, dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for s_ in s_in:
                s_.wait_stream(stream)
            pipeline(args.steps, download_grads)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            barrier(world, dev)
            return max_over_ranks(e0.elapsed_time(e1), world, dev) / args.steps

        def upload_alone(reps=10):
            """The step's host->device copies alone (no kernels): the bound the
            host link puts on the end-to-end step."""
            def once():
                for d_, h_ in zip(d_in[1], h_in):
                    for j, dp, hp in pieces(d_, h_):
                        with torch.cuda.stream(s_in[j]):
                            dp.copy_(hp, non_blocking=True)
            once()
            torch.cuda.synchronize(dev)
            u0 = torch.cuda.Event(enable_timing=True)
            u1 = torch.cuda.Event(enable_timing=True)
            u0.record(stream)
            for s_ in s_in:
                s_.wait_stream(stream)
            for _ in range(reps):
                once()
            for s_ in s_in:
                stream.wait_stream(s_)
            u1.record(stream)
            torch.cuda.synchronize(dev)
            return u0.elapsed_time(u1) / reps

        e2e_ms = timed_pipeline(False)
        e2e_grads_ms = timed_pipeline(True)
        up_ms = upload_alone()
        e2e = {"value": round(N * world / (e2e_ms * 1e-3) / 1e6, 3), "unit": "Mpoints/s",
               "ms_per_step": round(e2e_ms, 4), "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(h_loss[0].numel() * h_loss[0].element_size()),
               "result": "the loss <G, pyramid> (G is its gradient); point gradients stay on the device",
               "overlap": "double-buffered: uploads on %d copy stream(s) overlap the kernels" % n_cs,
               "upload_alone_ms": round(up_ms, 4),
               "upload_gbs": round(h2d / (up_ms * 1e-3) / 1e9, 1),
               "frac_of_upload_bound": round(up_ms / e2e_ms, 3),
               "with_gradients_downloaded": {
                   "value": round(N * world / (e2e_grads_ms * 1e-3) / 1e6, 3), "ms_per_step": round(e2e_grads_ms, 4),
                   "d2h_bytes_per_step": int(d2h_grads + 4)}}

    # forward-only time (same frame, no backward), for the forward ms/frame figure
    torch.cuda.synchronize(dev)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        r.project(pos, sw, ws, records=rec)
        r.splat_forward(rec, op, ws)
        r.blend(rec, op, desc, ws, pyramid=pyr)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    fwd_ms = max_over_ranks(f0.elapsed_time(f1), world, dev) / args.steps
    flags = r.status(ws)

    # the plain float32 form of a bfloat16 workload: the same step with float32 descriptors
    f32_form = None
    if b == 2 and not args.no_extras:
        rf = Renderer(sc.camera, sc.n_layers, K=sc.K, D=sc.D, desc_dtype=torch.float32, mode=args.mode,
                      tile=(tw, th), device=dev)
        desc32 = desc.to(torch.float32).contiguous()

        def step32():
            rf.project(pos, sw, ws, records=rec)
            rf.splat_forward(rec, op, ws)
            _, k32, n32, _, _ = rf.blend(rec, op, desc32, ws, store_lists=store, pyramid=pyr)
            rf.splat_backward(rec, op, desc32, G, ws, k32 if store else None, n32 if store else None, grads=grads)

        for _ in range(args.warmup):
            step32()
        torch.cuda.synchronize(dev)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(args.steps):
            step32()
        q1.record(stream)
        torch.cuda.synchronize(dev)
        ms32 = max_over_ranks(q0.elapsed_time(q1), world, dev) / args.steps
        f32_form = {"ms_per_step": round(ms32, 4), "bf16_speedup": round(ms32 / ms_per_step, 3)}
        del desc32

    # the same step with coarse-layer inclusion (Sec. 3.6): lists also hold the
    # fragments of the coarser pixels above; the blend runs layer by layer
    inclusion = None
    if not args.no_extras and not store:
        rc = Renderer(sc.camera, sc.n_layers, K=sc.K, D=sc.D, desc_dtype=desc_dtype, mode=args.mode,
                      tile=(tw, th), device=dev, coarse=True)
        ws_c = rc.new_workspace(N)

        def step_c():
            rc.project(pos, sw, ws_c, records=rec)
            rc.splat_forward(rec, op, ws_c)
            rc.blend(rec, op, desc, ws_c, pyramid=pyr)
            rc.splat_backward(rec, op, desc, G, ws_c, grads=grads)

        def timed(fn):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize(dev)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(args.steps):
                fn()
            a1.record(stream)
            torch.cuda.synchronize(dev)
            return max_over_ranks(a0.elapsed_time(a1), world, dev) / args.steps

        ms_c = timed(step_c)
        fwd_c = timed(lambda: (rc.project(pos, sw, ws_c, records=rec), rc.splat_forward(rec, op, ws_c),
                               rc.blend(rec, op, desc, ws_c, pyramid=pyr)))
        inclusion = {"ms_per_step": round(ms_c, 4), "overhead_ms": round(ms_c - ms_per_step, 4),
                     "forward_ms": round(fwd_c, 4), "forward_overhead_ms": round(fwd_c - fwd_ms, 4),
                     "flags": rc.status(ws_c), "workspace_bytes": int(ws_c.numel())}
        del ws_c

    camera = merge = size_init = None
    if not args.no_extras:
        # camera adjoint of the same frame (one pass over the points' gradients;
        # not part of the step): records, positions and point gradients read once
        cam_out = torch.empty(16, dtype=torch.float64, device=dev)
        r.camera_backward(pos, rec, grads[0], grads[1], out=cam_out)
        torch.cuda.synchronize(dev)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.steps):
            r.camera_backward(pos, rec, grads[0], grads[1], out=cam_out)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        cam_ms = max_over_ranks(c0.elapsed_time(c1), world, dev) / args.steps
        cam_bytes = 44 * N + 16 * 8
        camera = {"ms": round(cam_ms, 4), "algorithmic_bytes": cam_bytes,
                  "achieved_gbs": round(cam_bytes / (cam_ms * 1e-3) / 1e9, 1),
                  "frac": round(cam_bytes / (cam_ms * 1e-3) / 1e9 / peak, 4)}

        # pyramid merge of the frame into one image, and its adjoint (not part of the step)
        P0 = r.layer_offsets[1]
        Plast = P - r.layer_offsets[-2]
        merged = torch.empty((P, D), device=dev)
        g_img = (torch.rand((P0, D), generator=gen, device=dev) * 2 - 1).contiguous()
        g_pyr = torch.empty((P, D), device=dev)
        r.merge(pyr, out=merged)
        r.merge_backward(g_img, out=g_pyr)
        torch.cuda.synchronize(dev)
        m0, m1, m2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        m0.record(stream)
        for _ in range(args.steps):
            r.merge(pyr, out=merged)
        m1.record(stream)
        for _ in range(args.steps):
            r.merge_backward(g_img, out=g_pyr)
        m2.record(stream)
        torch.cuda.synchronize(dev)
        mf_ms = max_over_ranks(m0.elapsed_time(m1), world, dev) / args.steps
        mb_ms = max_over_ranks(m1.elapsed_time(m2), world, dev) / args.steps
        mf_bytes = 4 * D * (3 * P - P0)       # read P, write M, read each coarser merged layer once
        mb_bytes = 4 * D * (P0 + 2 * P - Plast)  # copy the image gradient, read each finer layer, write each layer
        # point-size initialisation of the cloud (exact 4-NN mean distance; not part of the step)
        from paper_2401_06003_gb300 import init_point_sizes
        sizes0 = torch.empty(N, device=dev)
        kws = torch.empty(int(r.lib.tp_init_sizes_workspace_bytes(N)), dtype=torch.uint8, device=dev)
        init_point_sizes(pos, out=sizes0, ws=kws)
        torch.cuda.synchronize(dev)
        k0, k1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        reps = max(1, min(args.steps, 5))
        k0.record(stream)
        for _ in range(reps):
            init_point_sizes(pos, out=sizes0, ws=kws)
        k1.record(stream)
        torch.cuda.synchronize(dev)
        knn_ms = max_over_ranks(k0.elapsed_time(k1), world, dev) / reps
        # algorithmic bytes: read every position once (12 N) and write every size (4 N);
        # the search itself is hash-grid lookups and distance arithmetic
        knn_bytes = 16 * N
        size_init = {"ms": round(knn_ms, 3), "mpoints_s": round(N / (knn_ms * 1e-3) / 1e6, 1), "k": 4,
                     "workspace_mb": round(kws.numel() / 1e6, 1), "algorithmic_bytes": knn_bytes,
                     "frac": round(knn_bytes / (knn_ms * 1e-3) / 1e9 / peak, 5),
                     "bound": "latency (random hash-grid lookups) and ALU, not HBM"}
        del kws

        fused = sc.camera.width * sc.camera.height * D <= (1 << 23)  # tp_merge's one-launch form
        merge = {"launches": 1 if fused else sc.n_layers, "backward_launches": sc.n_layers - 1,
                 "ms": round(mf_ms, 4),
                 "algorithmic_bytes": mf_bytes,
                 "frac": round(mf_bytes / (mf_ms * 1e-3) / 1e9 / peak, 4),
                 "backward_ms": round(mb_ms, 4), "backward_algorithmic_bytes": mb_bytes,
                 "backward_frac": round(mb_bytes / (mb_ms * 1e-3) / 1e9 / peak, 4)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc, args.cpu_frames, args.workload, N)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Mpoints/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if b == 4 else "f32 (bf16 descriptors)",
            "data": "synthetic",
            "config": {"workload": args.workload, "points": N, "width": sc.camera.width,
                       "height": sc.camera.height, "layers": sc.n_layers, "K": sc.K, "D": D,
                       "desc_dtype": "bf16" if b == 2 else "f32",
                       "mode": args.mode, "tile": args.tile, "parallelism": f"replicas{world}",
                       "point_order": order["kind"],
                       "l2": f"inputs larger than L2 ({(20 + b * D) * N / 1e6:.0f} MB of point inputs per step); "
                             "no flush"},
            "forward_ms": round(fwd_ms, 4), "fwd_bwd_ms": round(ms_per_step, 4),
            "forward_mpoints_s": round(N / (fwd_ms * 1e-3) / 1e6, 3),
            "counters": {"N": N, "V": V, "F": F, "Fk": Fk, "P": P},
            "roofline": roofline, "point_order": order, "camera_backward": camera, "pyramid_merge": merge,
            "point_size_init": size_init,
            "f32_form": f32_form, "accuracy": accuracy_report(args.workload) if b == 2 else None,
            "coarse_inclusion": inclusion,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": KERNELS_PER_STEP * args.steps, "clocks": clk, "device_flags": flags,
        }
        if world == 1 and not args.no_extras and not args.no_other_workloads and args.workload == "ground6m_1080p" \
                and not args.points:
            line["other_workloads"] = other_workloads(args)
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# batched multi-view (16 orbit cameras of uneven resolution, one graph)
# ---------------------------------------------------------------------------

def run_batch(args):
    import torch

    from paper_2401_06003_gb300 import BatchRenderer, Renderer, autotune_batch_tiles, scenes
    from paper_2401_06003_gb300.build import build as build_lib

    build_lib()
    rank, world, local = dist_setup(True)
    dev = torch.device("cuda", local)
    sc = scenes.make_config(args.workload, n=args.points or None)
    N, D, V = sc.n, sc.D, len(sc.cameras)
    pos = torch.from_numpy(sc.pos).to(dev)
    sw = torch.from_numpy(sc.size_w).to(dev)
    op = torch.from_numpy(sc.opacity).to(dev)
    desc = torch.from_numpy(sc.desc).to(dev)
    if args.point_order == "spatial":
        from paper_2401_06003_gb300 import permute_rows, spatial_order

        perm = spatial_order(pos)
        pos, sw, op, desc = (permute_rows(t, perm) for t in (pos, sw, op, desc))
    t0 = time.perf_counter()
    tiles, tuning = autotune_batch_tiles(sc.cameras, sc.n_layers, pos, sw, op, desc, K=sc.K, device=dev)
    tune_s = time.perf_counter() - t0
    br = BatchRenderer(sc.cameras, sc.n_layers, K=sc.K, D=D, tiles=tiles, device=dev)
    ws = br.new_workspace(N)
    rec = torch.empty((V, N, 4), device=dev)
    pyr = torch.empty((br.P, D), device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(4321 + rank)
    G = (torch.rand((br.P, D), generator=gen, device=dev) * 2 - 1).contiguous()
    grads = (torch.empty((N, 4), device=dev), None, torch.empty((N,), device=dev),  # packed (X, Y, Z, s_w) rows
             torch.empty((N, D), device=dev))

    def step():
        br.project(pos, sw, ws, records=rec)
        br.splat_forward(rec, op, ws)
        br.blend(rec, op, desc, ws, pyramid=pyr)
        br.splat_backward(rec, op, desc, G, ws, grads=grads)

    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(args.warmup):
            step()
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize(dev)
    if br.status(ws):
        raise RuntimeError("device status flags set after warm-up")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(2):
        graph.replay()
    stream = torch.cuda.current_stream(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device()) if not args.no_clocks else None
    barrier(world, dev)
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.start()
        time.sleep(0.3)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for s_ in range(args.steps):
        evs[s_][0].record(stream)
        graph.replay()
        evs[s_][1].record(stream)
    a1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    clk = clocks.stop() if clocks else None
    total_ms = max_over_ranks(a0.elapsed_time(a1), world, dev)
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    ms_per_step = total_ms / args.steps
    value = V * N * world / (ms_per_step * 1e-3) / 1e6

    # context for the batch: each view rendered alone (forward + backward), same tiles
    per_view = []
    for v, cam in enumerate(sc.cameras):
        r = Renderer(cam, sc.n_layers, K=sc.K, D=D, tile=tiles[v], device=dev)
        wsv = r.new_workspace(N)
        recv = torch.empty((N, 4), device=dev)
        pyrv = torch.empty((r.P, D), device=dev)
        Gv = br.view(G, v).contiguous()
        times = []
        for it in range(args.warmup + args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r.project(pos, sw, wsv, records=recv)
            r.splat_forward(recv, op, wsv)
            r.blend(recv, op, desc, wsv, pyramid=pyrv)
            r.splat_backward(recv, op, desc, Gv, wsv, grads=grads)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if it >= args.warmup:
                times.append(e0.elapsed_time(e1))
        per_view.append({"view": v, "width": cam.width, "height": cam.height, "tile": list(tiles[v]),
                         "p50_ms": round(float(np.percentile(times, 50)), 4),
                         "p99_ms": round(float(np.percentile(times, 99)), 4)})
        del wsv, recv, pyrv
    if rank == 0:
        line = {
            "metric": "batched multi-view fwd+bwd: aggregate Mpoints/s (views x points), 16 orbit views",
            "value": round(value, 3), "unit": "Mpoints/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "points": N, "views": V,
                       "resolutions": [[c.width, c.height] for c in sc.cameras], "layers": sc.n_layers,
                       "K": sc.K, "D": D, "mode": "recompute", "graph": "one CUDA graph per fwd+bwd batch step",
                       "point_order": args.point_order,
                       "l2": "inputs larger than L2; no flush"},
            "batch_step_ms": {"p50": round(float(np.percentile(step_ms, 50)), 4),
                              "p99": round(float(np.percentile(step_ms, 99)), 4)},
            # inside the batch every stage is one launch over all views, so each
            # view's outputs are complete when the step's last launch ends: a
            # view's latency in the batch is the batch step's (events per replay)
            "per_view_in_batch_ms": {"p50": round(float(np.percentile(step_ms, 50)), 4),
                                     "p99": round(float(np.percentile(step_ms, 99)), 4),
                                     "amortised": round(ms_per_step / V, 4)},
            # context: each view rendered alone with the same tiles (not a batch measurement)
            "single_view": per_view,
            "single_view_p50_ms": round(float(np.percentile([p["p50_ms"] for p in per_view], 50)), 4),
            "single_view_p99_ms": round(float(np.percentile([p["p99_ms"] for p in per_view], 99)), 4),
            "sum_of_single_view_p50_ms": round(sum(p["p50_ms"] for p in per_view), 4),
            "autotune": {"seconds": round(tune_s, 2),
                         "ms_by_resolution": {f"{w}x{h}": {f"{a}x{b}": round(t, 4) for (a, b), t in d.items()}
                                              for (w, h), d in tuning.items()}},
            "gpu_launches": 6 * args.steps, "clocks": clk,
        }
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the CPU oracle (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def _oracle_frame_fwd_bwd(sc, G_seed=1):
    import oracle

    fr = oracle.Frame.from_scene(sc)
    fr.render()
    G = np.random.default_rng(G_seed).uniform(-1, 1, (fr.n_pix, sc.D))
    fr.backward(G)


def _band_worker(workload, n, band, n_bands, G_seed, cmd_q, res_q):
    """One process of the multi-core oracle: the frame's pyramid rows
    [band P / n_bands, (band + 1) P / n_bands), rendered and back-propagated
    by the oracle as it stands, once per command.  The per-band gradients sum
    to the frame's (the loss is a sum over pixels)."""
    import oracle
    from paper_2401_06003_gb300 import scenes

    oracle.build()
    sc = scenes.make_config(workload, n=n)
    cam = sc.camera
    P = int(oracle.pyramid_layout(cam.width, cam.height, sc.n_layers)[0][-1])
    edges = np.linspace(0, P, n_bands + 1).astype(np.int64)
    pix = np.arange(edges[band], edges[band + 1], dtype=np.int64)
    G = np.random.default_rng(G_seed).uniform(-1, 1, (P, sc.D))[pix]
    res_q.put(("ready", band))
    while cmd_q.get() is not None:
        t = time.perf_counter()
        fr = oracle.Frame.from_scene(sc, pixels=pix)
        fr.render()
        fr.backward(G)
        del fr
        res_q.put(("done", time.perf_counter() - t))


class OraclePool:
    """The float64 oracle on every host core: one process per core, each on its
    own band of pyramid rows of the full frame.  Started with the spawn method
    (the parent may hold a CUDA context)."""

    def __init__(self, workload, n, workers):
        import multiprocessing as mp

        ctx = mp.get_context("spawn")
        self.res_q = ctx.Queue()
        self.cmd_qs = [ctx.Queue() for _ in range(workers)]
        self.procs = [ctx.Process(target=_band_worker, args=(workload, n, b, workers, 1, self.cmd_qs[b], self.res_q),
                                  daemon=True) for b in range(workers)]
        for p in self.procs:
            p.start()
        for _ in range(workers):
            kind, _ = self.res_q.get(timeout=600)
            assert kind == "ready"
        self.workers = workers

    def frame(self):
        """Wall seconds of one full frame (render + backward) over all workers."""
        t = time.perf_counter()
        for q in self.cmd_qs:
            q.put(1)
        for _ in range(self.workers):
            kind, _ = self.res_q.get(timeout=600)
            assert kind == "done"
        return time.perf_counter() - t

    def close(self):
        for q in self.cmd_qs:
            q.put(None)
        for p in self.procs:
            p.join(timeout=60)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(sc, frames, workload, n):
    """The float64 oracle, as it stands, on the full frame: once on one core
    and `frames` times on every host core (one process per core)."""
    import oracle

    oracle.build()
    t = time.perf_counter()
    _oracle_frame_fwd_bwd(sc)
    single = time.perf_counter() - t
    cores = host_cores()
    pool = OraclePool(workload, n, cores)
    try:
        dt = float(np.median([pool.frame() for _ in range(frames)]))
    finally:
        pool.close()
    return {"value": round(sc.n / dt / 1e6, 4), "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
            "sample": f"{frames} full frames of {sc.name} (fwd+bwd, float64 oracle), each split into {cores} bands "
                      f"of pyramid rows, one process per host core",
            "seconds_per_frame": round(dt, 3),
            "single_core": {"value": round(sc.n / single / 1e6, 4), "seconds_per_frame": round(single, 3)}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2401_06003_gb300 import scenes

    oracle.build()
    sc = scenes.make_config(args.workload, n=args.points or None)
    cores = host_cores()
    pool = OraclePool(args.workload, sc.n, cores)
    try:
        for _ in range(args.warmup):
            pool.frame()
        times = [pool.frame() for _ in range(args.steps)]
    finally:
        pool.close()
    ms = 1e3 * float(np.mean(times))
    value = sc.n / (ms * 1e-3) / 1e6
    sample = (f"full frames of {sc.name} (fwd+bwd, float64 oracle), each split into {cores} bands of pyramid rows, "
              f"one process per host core")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Mpoints/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "points": sc.n, "width": sc.camera.width,
                   "height": sc.camera.height, "layers": sc.n_layers, "K": sc.K, "D": sc.D,
                   "mode": "full lists (oracle)", "parallelism": f"cpu{cores}"},
        "cpu_baseline": {"value": round(value, 4), "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def other_workloads(args):
    """One-line summaries of the batched 16-view workload and the 4K bf16 workload,
    each run as its own bench process after the headline has been timed (the same
    timing rules; their full lines come from --workload)."""
    out = {}
    for w in ("ground6m_orbit16", "ground10m_4k_bf16"):
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", w, "--steps", str(args.steps),
               "--warmup", str(args.warmup), "--no-cpu-baseline", "--no-e2e"]
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            d = json.loads(r.stdout.strip().splitlines()[-1])
        except (subprocess.SubprocessError, ValueError, IndexError) as exc:
            out[w] = {"error": str(exc)[:200]}
            continue
        keep = ("metric", "value", "unit", "ms_per_step", "forward_ms", "batch_step_ms", "per_view_in_batch_ms",
                "single_view_p50_ms", "single_view_p99_ms", "f32_form", "clocks", "device_flags")
        s = {k: d[k] for k in keep if k in d}
        if d.get("roofline"):
            s["roofline_frac"] = d["roofline"].get("frac")
            s["step_frac"] = d["roofline"].get("step", {}).get("frac")
        acc = d.get("accuracy")
        if acc:  # max relative errors on the crops against the float64 oracle
            s["accuracy_max_rel"] = {q: {k: acc[q][k]["max_rel"] for k in ("vs_oracle_bf16_values",
                                                                            "vs_oracle_f32_values")}
                                     for q in ("pyramid", "grad_pos", "grad_size_w", "grad_opacity", "grad_desc")
                                     if q in acc}
        out[w] = s
    return out


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.endswith("orbit16"):
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
