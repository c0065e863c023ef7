#!/usr/bin/env python
"""Benchmark: rasterization + micro-edge backward throughput (Mpix/s) on GB300.

Workload (default): the multi-view head scene -- a 65,538-vertex / 131,072-triangle
displaced sphere with a 1024^2 bilinear texture seen by 32 cameras at 1334x2048
(87.4 Mpix per step), channels RGB + mask + depth, upstream gradient N(0,1).
One step = project -> bin + raster -> shade -> fused edge + interior backward ->
projection backward, i.e. the whole forward+backward path, all views at once.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on
the host cores instead (bounded sample of the same workload).
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
sys.path.insert(0, ROOT)

METRIC = "raster+micro-edge backward Mpix/s on 1 GB300; % HBM roofline; batched vs plain"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", type=int, default=32)
    ap.add_argument("--views", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def backward_bytes_per_launch(n, H, W, C, V):
    """Algorithmic bytes of the fused backward kernel: per pixel the index (4 B), the image and its
    gradient (4C + 4C B); per (view, vertex) the vertex record (32 B) and the gradient (12 B)."""
    return n * H * W * (4 + 8 * C) + n * V * (32 + 12)


def step_bytes(n, H, W, C, V, T, tex_bytes):
    """Algorithmic bytes of one whole step (all kernels): see the design notes."""
    fwd = n * H * W * (4 + 4 + 4 * C) + n * T * 12 + n * V * 32 + V * 12 + tex_bytes
    bwd = n * H * W * (4 + 8 * C) + n * V * (32 + 12) + V * 12
    return fwd + bwd


# ---------------------------------------------------------------------------
# CPU oracle arm
# ---------------------------------------------------------------------------

def oracle_sample(scene, n_views: int, threads: int):
    import oracle

    views = list(range(n_views))
    g = [np.random.default_rng(100 + v).standard_normal((scene.H, scene.W, scene.shading.C), dtype=np.float32)
         for v in views]
    t0 = time.perf_counter()
    res = oracle.render(scene, views, threads=threads)
    oracle.backward_scene(scene, res, g, views, threads=threads)
    dt = time.perf_counter() - t0
    return n_views * scene.H * scene.W / dt / 1e6, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2405_02508_gb300 import scenes

    scene = scenes.head_multiview(n_views=args.views)
    threads = min(os.cpu_count() or 1, 16, args.views)
    for _ in range(args.warmup):
        oracle_sample(scene, threads, threads)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_sample(scene, threads, threads)
        times.append(dt)
    px = threads * scene.H * scene.W
    value = px * len(times) / sum(times) / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"head multi-view {args.views}x{scene.W}x{scene.H}, 131072 tris, RGB+mask+depth",
                   "sample": f"{threads} of {args.views} views per step"},
        "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": threads, "kind": "oracle",
                         "sample": f"{threads} full-size views per step, one thread per view"},
        "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300 import scenes
    from paper_2405_02508_gb300.render import Renderer

    B.lib()
    dev = "cuda"
    # weak scaling: every rank renders its own batch of views (cameras drawn with a rank-specific seed)
    scene = scenes.head_multiview(n_views=args.views, seed=6 + rank)
    n, H, W, C = scene.n_views, scene.H, scene.W, scene.shading.C
    V, T = len(scene.verts), len(scene.tris)
    verts = torch.from_numpy(scene.verts).to(dev)
    cams = B.cameras_tensor(scene.cams)
    attr = torch.from_numpy(scene.attr).to(dev)
    tex = torch.from_numpy(scene.tex).to(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7 + rank)
    g = torch.randn((n, H, W, C), generator=gen, device=dev, dtype=torch.float32)
    r = Renderer(torch.from_numpy(scene.tris), V, n, H, W, scene.shading, attr.shape[1], tex.shape, tile=args.tile)
    r.forward(verts, cams, attr, tex, checked=True)  # sizes the bin list once
    stream = torch.cuda.current_stream()

    ev_b0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_b1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_r0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_r1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    def step(i=None):
        if i is not None:
            ev_r0[i].record(stream)
        r.project(verts, cams)
        r.rasterize(checked=False)
        if i is not None:
            ev_r1[i].record(stream)
        r.shade(attr, tex)
        r.grad_vpix.zero_()
        r.grad_verts.zero_()
        if i is not None:
            ev_b0[i].record(stream)
        B.mer_backward(r.vpix, r.tris, r.index, r.image, g, attr, tex, r.sh, B.MER_EDGE | B.MER_INTERIOR |
                       B.MER_INTERSECT, r.grad_vpix, None, r.workspace)
        if i is not None:
            ev_b1[i].record(stream)
        B.mer_project_backward(cams, r.vpix, r.grad_vpix, r.grad_verts)

    for _ in range(args.warmup):
        step()
    r.check_status()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(i)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    r.check_status()
    ms = t0.elapsed_time(t1) / args.steps
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    bwd_ms = float(np.mean([a.elapsed_time(b) for a, b in zip(ev_b0, ev_b1)]))
    ras_ms = float(np.mean([a.elapsed_time(b) for a, b in zip(ev_r0, ev_r1)]))

    # end-to-end: host vertex positions in, host vertex gradients out, copies inside the timed region
    h_verts = torch.from_numpy(scene.verts).pin_memory()
    h_grad = torch.empty((V, 3), dtype=torch.float32).pin_memory()
    d_verts = torch.empty_like(verts)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        d_verts.copy_(h_verts, non_blocking=True)
        r.project(d_verts, cams)
        r.rasterize(checked=False)
        r.shade(attr, tex)
        r.grad_vpix.zero_()
        r.grad_verts.zero_()
        B.mer_backward(r.vpix, r.tris, r.index, r.image, g, attr, tex, r.sh, 7, r.grad_vpix, None, r.workspace)
        B.mer_project_backward(cams, r.vpix, r.grad_vpix, r.grad_verts)
        h_grad.copy_(r.grad_verts, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        tt = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item())

    px_step = n * H * W * world
    value = px_step / (ms * 1e-3) / 1e6
    peak, peak_kind = peaks()
    bb = backward_bytes_per_launch(n, H, W, C, V)
    achieved = bb / (bwd_ms * 1e-3) / 1e9
    launches_per_step = 10  # project 1, binning+scan+raster 6, shade 1, backward 1, projection backward 1
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"head multi-view: {n} views x {W}x{H}, {V} verts / {T} tris, 1024^2 texture, "
                               f"RGB+mask+depth (C={C}), upstream N(0,1)", "views_per_gpu": n, "H": H, "W": W,
                   "triangles": T, "tile": args.tile, "l2": "inputs larger than L2 (images 1.7 GB per step)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "kernel": "k_backward (fused edge + interior)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "peak_kind": peak_kind, "kernel_ms": bwd_ms, "algorithmic_bytes": bb},
        "kernels_ms": {"project+bin+raster": ras_ms, "backward": bwd_ms},
        "step_algorithmic_gbs": step_bytes(n, H, W, C, V, T, tex.numel() * 4) / (ms * 1e-3) / 1e9,
        "e2e": {"value": px_step / (e2e_ms * 1e-3) / 1e6, "unit": "Mpix/s", "h2d_bytes_per_step": V * 12,
                "d2h_bytes_per_step": V * 12, "ms_per_step": e2e_ms},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = min(os.cpu_count() or 1, 8)
        v, dt = oracle_sample(scene, threads, threads)
        line["cpu_baseline"] = {"value": v, "unit": "Mpix/s", "cores": threads, "kind": "oracle",
                                "sample": f"{threads} of {n} full-size views, one thread each ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
