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
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", type=int, default=0, help="bin tile; 0 = autotune over 16/32/64")
    ap.add_argument("--views", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the per-view launch path")
    ap.add_argument("--workload", default="multiview", choices=["multiview", "uneven", "configs"],
                    help="multiview: 32 views of the head mesh (default); uneven: 256-mesh Adam fitting loop; "
                         "configs: one line per single-view config (tiny, intersection, head-scale) with the "
                         "batched and per-view paths and the oracle on 1 and all host threads")
    ap.add_argument("--items", type=int, default=256)
    ap.add_argument("--fit-steps", type=int, default=200, help="uneven workload: Adam steps of the RMSE runs")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload: skip the side table of the single-view configurations")
    ap.add_argument("--split-views", action="store_true",
                    help="N > 1: split the 32 views of the one mesh over the ranks and sum the vertex gradient "
                         "over the ranks every step (strong scaling); default: every rank its own 32 views")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 50 ms while the timed region runs."""

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
                                          "--format=csv,noheader,nounits", "-lms", "50"],
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


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) and warp instructions (smsp__inst_executed.sum) of
# one k_backward_batch launch, from an ncu capture of the same workload at 4 views (inputs already larger than
# L2), per pixel of the launch, with the sha256 of the kernel's sources they were taken on: a launch of n views
# moves / issues n*H*W times these.  They are reported only while the sources are unchanged.
BACKWARD_TRAFFIC = {"bytes_per_pixel": 24.4699, "warp_instructions_per_pixel": 31.0864,
                    "sources_sha256": "6c09ff0940653e50a07548f9ec794d428185f7d555c26de972205dd402d7dd76",
                    "profile": "profiles/ncu_k_backward_batch_head_4x1334x2048.md"}


def backward_sources_sha256() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in ("backward.cu", "mer_device.cuh"):
        with open(os.path.join(ROOT, "paper_2405_02508_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def backward_traffic(pixels: int):
    t = BACKWARD_TRAFFIC
    if t["bytes_per_pixel"] is None or t["sources_sha256"] != backward_sources_sha256():
        return None
    return t["bytes_per_pixel"] * pixels


def issue_peak() -> float:
    """Warp instructions per second the SMs can issue: one per scheduler (4 per SM) per cycle at the GPU's
    maximum SM clock."""
    import torch

    props = torch.cuda.get_device_properties(0)
    mhz = 2070.0
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=10).stdout.split()
        mhz = float(out[0])
    except Exception:
        pass
    return props.multi_processor_count * 4 * mhz * 1e6


def backward_issue_roofline(pixels: int, kernel_ms: float):
    """Second roofline of the backward: warp instructions per launch (ncu count per pixel x pixels, null once
    the sources changed) over the issue peak."""
    t = BACKWARD_TRAFFIC
    if t.get("warp_instructions_per_pixel") is None or t["sources_sha256"] != backward_sources_sha256():
        return None
    inst = t["warp_instructions_per_pixel"] * pixels
    peak = issue_peak()
    achieved = inst / (kernel_ms * 1e-3)
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp instructions/s",
            "frac": achieved / peak, "instructions": inst,
            "peak_kind": "derived: SMs x 4 schedulers x 1 instruction per cycle x max SM clock"}


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


def band_scene(scene, y0: int, rows: int):
    """The same views restricted to rows [y0, y0 + rows): the principal point moves up by y0, so the band's
    pixels are exactly those of the full view."""
    import dataclasses

    cams = scene.cams.copy()
    cams["cy"] = cams["cy"] - y0
    return dataclasses.replace(scene, cams=cams, H=rows)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2405_02508_gb300 import scenes

    scene = scenes.head_multiview(n_views=args.views)
    threads = min(os.cpu_count() or 1, args.views)
    rows = 128  # each step: one 128-row band of `threads` views, the band moving down the image step by step
    bands = [band_scene(scene, y0, rows) for y0 in range(0, scene.H, rows)]
    for k in range(args.warmup):
        oracle_sample(bands[k % len(bands)], threads, threads)
    times = []
    for k in range(args.steps):
        _, dt = oracle_sample(bands[k % len(bands)], threads, threads)
        times.append(dt)
    px = threads * rows * scene.W
    value = px * len(times) / sum(times) / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"head multi-view {args.views}x{scene.W}x{scene.H}, 131072 tris, RGB+mask+depth",
                   "sample": f"a {rows}-row band of {threads} of the {args.views} views per step"},
        "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": threads, "kind": "oracle",
                         "sample": f"{rows}-row bands (1334 x {rows} px) of {threads} views per step, one thread "
                                   "per view, the band moving down the full 2048-row views"},
        "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_uneven(args):
    """Uneven batch: 256 meshes (500..200k triangles, 128^2..1024^2) per GPU, Adam steps of the mask + normal
    fit.  With N ranks the batch has N x 256 meshes, split by longest-processing-time on T + H*W.  Besides the
    step throughput: the backward's roofline, the per-item launch path on the same render + backward, and the
    vertex RMSE after --fit-steps steps of plain Adam and of the Laplacian-preconditioned loop; on one GPU the
    CPU baseline is the same plain-Adam loop driven by the FP64 oracle on four items of the batch (its RMSE
    over those items against the GPU loop's)."""
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300 import scenes, shard
    from paper_2405_02508_gb300.batch import PlainRenderer
    from paper_2405_02508_gb300.fit import UnevenFit

    world, rank, local = shard.env_ranks()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n_all = world * args.items
    nis, res = scenes.uneven_plan(n_all)
    costs = [shard.item_cost(8 * n * n, r, r) for n, r in zip(nis, res)]
    mine = shard.lpt_assign(costs, world)[rank]
    items = scenes.uneven_batch(n_items=n_all, subset=mine)
    fit = UnevenFit(items, tile=args.tile if args.tile > 0 else 32)
    stream = torch.cuda.current_stream()
    fit.run(args.warmup)
    torch.cuda.synchronize()
    shard.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fit.run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    shard.barrier()
    ms = shard.max_over_ranks(e0.elapsed_time(e1) / args.steps, "cuda")
    pixels = sum(it.H * it.W for it in items)
    all_pixels = sum(r * r for r in res)

    # the backward kernel of one step, timed on the launching stream, and its roofline
    br = fit.br
    x = fit.v_init.contiguous()
    nrm = fit._render(x)
    fit._l2()
    ga = torch.zeros_like(nrm)
    kb = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    bwd_ms = []
    for _ in range(5):
        br.grad_vpix.zero_()
        kb[0].record(stream)
        B.mer_batch_backward(br.vpix, br.tris, br.items, br.tot, br.index, br.image, fit._gimg, nrm, None, br.sh, 7,
                             br.grad_vpix, ga, br.workspace, br.persistent_ctas, br.cover)
        kb[1].record(stream)
        torch.cuda.synchronize()
        bwd_ms.append(kb[0].elapsed_time(kb[1]))
    bwd_ms = float(np.median(bwd_ms))
    C, Ca = br.C, 3
    V_rows = int(br.tot.vrecs)
    bb = pixels * (4 + 8 * C) + V_rows * (32 + 12) + sum(len(it.verts) for it in items) * 4 * Ca
    peak, peak_kind = peaks()

    # like for like, render + backward only (no normals, no Adam): the batched step against one launch
    # sequence per item
    g = fit._gimg
    gv_items = [g[br.item_pix[k][0]:br.item_pix[k][0] + it.H * it.W].view(1, it.H, it.W, C)
                for k, it in enumerate(items)]
    verts_items = [x[int(fit.vert_off[k]):int(fit.vert_off[k + 1])].contiguous() for k in range(len(items))]
    attr_items = [nrm[int(fit.vert_off[k]):int(fit.vert_off[k + 1])].contiguous() for k in range(len(items))]

    def batched_rb():
        br.forward(x, nrm)
        br.backward(g, nrm)

    plain_ms = batched_rb_ms = None
    if not args.no_plain:
        pr = PlainRenderer([(it.verts, it.tris) for it in items], [(k, k, it.H, it.W) for k, it in enumerate(items)],
                           np.concatenate([it.cams for it in items]), items[0].shading, Ca)
        pr.step(verts_items, attr_items, gv_items, None, checked=True)
        for fn, key in ((lambda: pr.step(verts_items, attr_items, gv_items, None), "plain"), (batched_rb, "batched")):
            fn()
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            t0.record(stream)
            for _ in range(reps):
                fn()
            t1.record(stream)
            torch.cuda.synchronize()
            if key == "plain":
                plain_ms = t0.elapsed_time(t1) / reps
            else:
                batched_rb_ms = t0.elapsed_time(t1) / reps
        del pr

    # vertex RMSE after --fit-steps steps: plain Adam (lr 1e-3) and the preconditioned loop (lambda 16)
    nsub = scenes.uneven_plan(n_all)[0]
    Tall = np.array([8 * n * n for n in nsub])
    order = np.argsort(Tall, kind="stable")
    sub_global = [int(order[0]), int(order[len(order) // 3]), int(order[2 * len(order) // 3]), int(order[-1])]
    sub = [mine.index(i) for i in sub_global if i in mine]  # positions of those items in this rank's batch
    v_adam = fit.run(args.fit_steps, lr=1e-3)
    v_adam4 = fit.run(args.fit_steps, lr=1e-4)
    v_pre = fit.run_preconditioned(args.fit_steps, lr=2e-3, lam=16.0)
    rmse = {"steps": args.fit_steps, "initial": fit.rmse(fit.v_init), "adam_lr1e-3": fit.rmse(v_adam),
            "adam_lr1e-4": fit.rmse(v_adam4), "preconditioned_lambda16_lr2e-3": fit.rmse(v_pre),
            "loss_initial": fit.loss(fit.v_init), "loss_adam_lr1e-3": fit.loss(v_adam),
            "loss_adam_lr1e-4": fit.loss(v_adam4), "loss_preconditioned": fit.loss(v_pre)}
    if sub:
        rmse.update(subset_items=[mine[k] for k in sub], subset_initial=fit.rmse(fit.v_init, sub),
                    subset_adam=fit.rmse(v_adam, sub))

    line = {"metric": METRIC, "value": all_pixels / (ms * 1e-3) / 1e6, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"uneven batch: {n_all} meshes, {sum(8 * n * n for n in nis)} tris, "
                                   f"{all_pixels / 1e6:.1f} Mpix per step; Adam lr 1e-3, mask + normal L2",
                       "step": "normals + batched render + micro-edge/interior backward + normals backward + Adam",
                       "parallelism": f"LPT shards x{world}, no collective"},
            "roofline": {"bound": "hbm", "kernel": "k_backward_batch (fused edge + interior, attribute gradients)",
                         "achieved": bb / (bwd_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": bb / (bwd_ms * 1e-3) / 1e9 / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel_ms": bwd_ms, "algorithmic_bytes": bb},
            "render_backward": None if plain_ms is None else
            {"batched_ms": batched_rb_ms, "plain_per_item_ms": plain_ms,
             "batched_mpix_s": pixels / (batched_rb_ms * 1e-3) / 1e6,
             "plain_mpix_s": pixels / (plain_ms * 1e-3) / 1e6, "plain_launch_sequences": len(items)},
            "rmse": rmse}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and sub:
        import time

        from oracle.fitloop import oracle_fit

        rows = np.concatenate([np.arange(fit.vert_off[k], fit.vert_off[k + 1]) for k in sub])
        sel = torch.from_numpy(rows).cuda()
        threads = os.cpu_count() or 1
        t0 = time.perf_counter()
        v_orc = oracle_fit([items[k] for k in sub], fit.v_init[sel].cpu().numpy(), args.fit_steps, lr=1e-3,
                           threads=threads)
        dt = time.perf_counter() - t0
        d = v_orc - fit.v_true[sel].cpu().numpy().astype(np.float64)
        rmse["subset_oracle_driven"] = float(np.sqrt((d ** 2).sum(axis=1).mean()))
        spx = sum(items[k].H * items[k].W for k in sub) * args.fit_steps
        line["cpu_baseline"] = {"value": spx / dt / 1e6, "unit": "Mpix/s", "cores": threads, "kind": "oracle",
                                "sample": f"the same Adam loop on items {rmse['subset_items']} of the batch, "
                                          f"{args.fit_steps} steps with oracle gradients ({dt:.0f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def config_table(args, with_oracle: bool = True) -> list[dict]:
    """The single-view configurations (tiny icosphere, interpenetrating spheres, head-scale view) through the
    batched graph path (bin tile and persistent grid autotuned per workload) and the per-view launch path,
    each with its algorithmic-byte roofline and the FP64 oracle on one host thread; for the two spheres also
    the intersection pairs' share of the differing pairs (oracle counts) and the backward with and without
    the intersection term (the paper's ablation)."""
    import time

    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300 import scenes
    from paper_2405_02508_gb300.batch import BatchRenderer, PlainRenderer, autotune, workload_key

    B.lib()
    cases = [("tiny icosphere 128x128, 1280 tris, RGB", scenes.tiny_icosphere()),
             ("two interpenetrating icospheres 512x512, 40960 tris, normals+mask+depth", scenes.two_spheres()),
             ("head-scale single view 1024x1024, 131072 tris, textured RGB+mask", scenes.head_single_view())]
    out = []
    for name, sc in cases:
        H, W, C = sc.H, sc.W, sc.shading.C
        verts = torch.from_numpy(sc.verts).cuda()
        attr = torch.from_numpy(sc.attr).cuda()
        tex = torch.from_numpy(sc.tex).cuda() if sc.tex is not None else None
        g = torch.from_numpy(sc.upstream()).cuda().reshape(-1, C)
        meshes, items = [(sc.verts, sc.tris)], [(0, 0, H, W)]

        def make(tile, ctas=0):
            r = BatchRenderer(meshes, items, sc.cams, sc.shading, sc.attr.shape[1], tex, tile=tile,
                              persistent_ctas=ctas)
            r.prepare(verts, attr, tex)
            return r

        tile, ctas, _ = autotune(make, lambda r: r.step(verts, attr, g, tex), key=workload_key(items, meshes))
        br = make(tile, ctas)
        br.capture(verts, attr, g, tex)
        pr = PlainRenderer(meshes, items, sc.cams, sc.shading, sc.attr.shape[1], None if tex is None else tex.shape,
                           tile=16)
        gv = [g.view(1, H, W, C)]
        pr.step([verts], [attr], gv, tex, checked=True)

        def timed(fn, reps):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        reps = max(args.steps, 20)
        ms_b = timed(br.replay, reps)
        ms_p = timed(lambda: pr.step([verts], [attr], gv, tex), reps)
        px = H * W
        fwd = px * (4 + 4 + 4 * C) + len(sc.tris) * 12 + len(sc.verts) * 32
        bwd = px * (4 + 8 * C) + len(sc.verts) * 44
        peak, kind = peaks()
        row = {"workload": name, "unit": "Mpix/s", "batched": px / (ms_b * 1e-3) / 1e6, "batched_ms": ms_b,
               "tile": tile, "persistent_ctas": br.persistent_ctas,
               "plain": px / (ms_p * 1e-3) / 1e6, "plain_ms": ms_p,
               "algorithmic_gbs": (fwd + bwd) / (ms_b * 1e-3) / 1e9,
               "roofline_frac": (fwd + bwd) / (ms_b * 1e-3) / 1e9 / peak, "peak_gbs": peak, "peak_kind": kind}
        if sc.name.startswith("two_spheres"):
            # intersections on / off (the paper's ablation): the batched backward alone, both term sets
            def bwd_terms(terms):
                def fn():
                    br.grad_vpix.zero_()
                    B.mer_batch_backward(br.vpix, br.tris, br.items, br.tot, br.index, br.image, g, attr, tex, br.sh,
                                         terms, br.grad_vpix, None, br.workspace, br.persistent_ctas, br.cover)
                return fn

            on, off = timed(bwd_terms(7), reps), timed(bwd_terms(3), reps)
            row["intersections"] = {"backward_ms_on": on, "backward_ms_off": off,
                                    "overhead": on / off - 1.0}
        if with_oracle:
            import oracle

            t0 = time.perf_counter()
            ov = oracle.render(sc, [0], threads=1)
            _, _, counts, _ = oracle.backward_scene(sc, ov, [sc.upstream()[0]], [0], threads=1)
            dt = time.perf_counter() - t0
            row["cpu_oracle_1thread"] = {"value": px / dt / 1e6, "unit": "Mpix/s", "seconds": dt}
            if "intersections" in row:
                c = counts[0]
                row["intersections"].update(pairs_differing=c["differing"], pairs_intersection=c["intersection"],
                                            pairs_overhang=c["overhang"],
                                            intersection_share=c["intersection"] / max(c["differing"], 1))
        out.append(row)
        del br, pr
        torch.cuda.empty_cache()
    return out


def run_configs(args):
    """Side table (one JSON line per configuration, see config_table), then the oracle on the two batched
    workloads: one view of the multi-view scene on one thread, and one full step over all 256 meshes of the
    uneven batch on all host threads."""
    import time

    import torch

    torch.cuda.set_device(0)
    for row in config_table(args):
        row["metric"] = METRIC
        print(json.dumps(row), flush=True)
    from paper_2405_02508_gb300 import scenes

    mv = scenes.head_multiview(n_views=1)
    v1, d1 = oracle_sample(mv, 1, 1)
    print(json.dumps({"workload": "head multi-view, 1 of 32 views 1334x2048", "cpu_oracle_1thread":
                      {"value": v1, "unit": "Mpix/s", "seconds": d1}}), flush=True)
    import oracle

    items = scenes.uneven_batch(n_items=args.items)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()

    def one(it):
        r = oracle.render(it)[0]
        g = it.upstream()[0]
        oracle.backward(r.scr, r.snap, r.flags, it.tris, r.index, r.image, g, it.attr, it.shading, want_attr=True)

    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, items))
    dt = time.perf_counter() - t0
    px = sum(it.H * it.W for it in items)
    print(json.dumps({"workload": f"uneven batch, one full step over {len(items)} meshes",
                      "cpu_oracle_all_threads": {"value": px / dt / 1e6, "unit": "Mpix/s", "seconds": dt,
                                                 "cores": threads}}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "uneven":
        run_uneven(args)
        return
    if args.workload == "configs":
        run_configs(args)
        return
    import torch
    import torch.distributed as dist

    from paper_2405_02508_gb300 import shard

    world, rank, local = shard.env_ranks()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300 import scenes
    from paper_2405_02508_gb300.batch import BatchRenderer, PlainRenderer, autotune, workload_key

    B.lib()
    dev = "cuda"
    split = args.split_views and world > 1
    if split:
        # strong scaling: the 32 views of one mesh split over the ranks; the vertex gradient is summed over
        # the ranks every step
        scene = scenes.head_multiview(n_views=args.views)
        my_views = shard.split_views(args.views, world)[rank]
    else:
        # weak scaling: every rank renders its own batch of views (cameras drawn with a rank-specific seed)
        scene = scenes.head_multiview(n_views=args.views, seed=shard.view_seed(6, rank))
        my_views = list(range(args.views))
    n, H, W, C = len(my_views), scene.H, scene.W, scene.shading.C
    V, T = len(scene.verts), len(scene.tris)
    verts = torch.from_numpy(scene.verts).to(dev)
    attr = torch.from_numpy(scene.attr).to(dev)
    tex = torch.from_numpy(scene.tex).to(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(shard.view_seed(7, 0 if split else rank))
    g = torch.randn((args.views * H * W, C), generator=gen, device=dev, dtype=torch.float32)
    if split:  # this rank's views' part of the upstream gradient of all views
        g = g.view(args.views, H * W, C)[my_views[0]:my_views[-1] + 1].reshape(-1, C).contiguous()
    meshes = [(scene.verts, scene.tris)]
    items = [(0, v, H, W) for v in my_views]
    stream = torch.cuda.current_stream()

    def make(tile, ctas=0):
        br = BatchRenderer(meshes, items, scene.cams, scene.shading, attr.shape[1], tex, tile=tile,
                           persistent_ctas=ctas)
        br.prepare(verts, attr, tex)
        return br

    if args.tile > 0:
        tile, ctas, tune = args.tile, 0, {}
    else:  # autotuned bin tile and persistent grid, cached per workload signature
        tile, ctas, tune = autotune(make, lambda r: r.step(verts, attr, g, tex), key=workload_key(items, meshes))
    br = make(tile, ctas)
    br.capture(verts, attr, g, tex)  # one CUDA graph: the whole forward + backward step

    for _ in range(args.warmup):
        br.replay()
    torch.cuda.synchronize()
    br.check()
    clocks = ClockSampler(local)
    clocks.start()
    shard.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        br.replay()
        if split:
            shard.sum_over_ranks(br.grad_verts)  # the gradient of all views on every rank
    t1.record(stream)
    torch.cuda.synchronize()
    shard.barrier()
    clk = clocks.stop()
    br.check()
    ms = shard.max_over_ranks(t0.elapsed_time(t1) / args.steps, dev)

    # per-kernel times: the same step run eagerly with CUDA events around the stages on the launching stream
    ev = {k: [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)] for k in ("fwd", "bwd", "rast")}
    for i in range(args.steps):
        ev["fwd"][2 * i].record(stream)
        B.mer_batch_project(verts, br.cams, br.items, br.tot, br.vpix)
        ev["rast"][2 * i].record(stream)
        B.mer_batch_render(br.vpix, br.tris, br.items, br.tot, br.workspace, br.index, attr, tex, br.bg, br.sh,
                           br.image, None, None, br.persistent_ctas, br.cover)
        ev["rast"][2 * i + 1].record(stream)
        ev["fwd"][2 * i + 1].record(stream)
        br.grad_vpix.zero_()
        br.grad_verts.zero_()
        ev["bwd"][2 * i].record(stream)
        B.mer_batch_backward(br.vpix, br.tris, br.items, br.tot, br.index, br.image, g, attr, tex, br.sh, 7,
                             br.grad_vpix, None, br.workspace, br.persistent_ctas, br.cover)
        ev["bwd"][2 * i + 1].record(stream)
        B.mer_batch_project_backward(br.cams, br.items, br.tot, br.vpix, br.grad_vpix, br.grad_verts)
    torch.cuda.synchronize()
    kms = {k: float(np.mean([e[2 * i].elapsed_time(e[2 * i + 1]) for i in range(args.steps)])) for k, e in ev.items()}

    # end-to-end through the public API: host vertex positions in, host vertex gradients out, per step
    h_verts = torch.from_numpy(scene.verts).pin_memory()
    h_grad = torch.empty((V, 3), dtype=torch.float32).pin_memory()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    shard.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        verts.copy_(h_verts, non_blocking=True)  # the graph reads `verts` in place
        br.replay()
        if split:
            shard.sum_over_ranks(br.grad_verts)
        h_grad.copy_(br.grad_verts[:V], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = shard.max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)

    # plain path: each view its own launch sequence (same kernels, no batching, no graph)
    plain_ms = None
    if not args.no_plain:
        pr = PlainRenderer(meshes, items, scene.cams, scene.shading, attr.shape[1], tex.shape, tile=32)
        gv = [g[k * H * W:(k + 1) * H * W].view(1, H, W, C) for k in range(n)]
        pr.step([verts], [attr], gv, tex, checked=True)
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(max(1, args.steps // 2)):
            pr.step([verts], [attr], gv, tex)
        p1.record(stream)
        torch.cuda.synchronize()
        plain_ms = p0.elapsed_time(p1) / max(1, args.steps // 2)
        del pr

    px_step = args.views * H * W * (1 if split else world)
    value = px_step / (ms * 1e-3) / 1e6
    peak, peak_kind = peaks()
    bb = backward_bytes_per_launch(n, H, W, C, V)
    achieved = bb / (kms["bwd"] * 1e-3) / 1e9
    launches_per_step = 9  # project 1, setup/count 1, scan 3, fill 1, raster+shade 1, backward 1, proj. backward 1
    scaling = "strong" if split else "weak"
    parallelism = (f"views split x{world}, vertex gradient summed over the ranks (all-reduce) each step" if split
                   else f"replicas x{world}")
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": scaling,
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"head multi-view: {n} views x {W}x{H}, {V} verts / {T} tris, 1024^2 texture, "
                               f"RGB+mask+depth (C={C}), upstream N(0,1)", "views_per_gpu": n, "H": H, "W": W,
                   "triangles": T, "path": "batched: persistent raster/backward over a device tile queue, "
                   "one CUDA graph per step", "tile": tile, "persistent_ctas": br.persistent_ctas, "autotune_ms (tile/ctas)": tune,
                   "l2": "inputs larger than L2 (images 1.7 GB per step)", "parallelism": parallelism},
        "roofline": {"bound": "hbm", "kernel": "k_backward_batch (fused edge + interior)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": backward_traffic(n * H * W),
                     "peak_kind": peak_kind, "kernel_ms": kms["bwd"], "algorithmic_bytes": bb},
        "roofline_issue": backward_issue_roofline(n * H * W, kms["bwd"]),
        "kernels_ms": {"forward (project+raster+shade)": kms["fwd"], "bin+raster+shade (fused)": kms["rast"],
                       "backward": kms["bwd"]},
        "step_algorithmic_gbs": step_bytes(n, H, W, C, V, T, tex.numel() * 4) / (ms * 1e-3) / 1e9,
        "plain": None if plain_ms is None else {"value": px_step / (plain_ms * 1e-3) / 1e6, "unit": "Mpix/s",
                                                "ms_per_step": plain_ms, "launches_per_step": 10 * n},
        "e2e": {"value": px_step / (e2e_ms * 1e-3) / 1e6, "unit": "Mpix/s", "h2d_bytes_per_step": V * 12,
                "d2h_bytes_per_step": V * 12, "ms_per_step": e2e_ms},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_configs:
        line["configs"] = config_table(args, with_oracle=not args.no_cpu_baseline)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = min(os.cpu_count() or 1, n)
        v, dt = oracle_sample(scene, threads, threads)
        line["cpu_baseline"] = {"value": v, "unit": "Mpix/s", "cores": threads, "kind": "oracle",
                                "sample": f"{threads} of {n} full-size views, one host thread each, every host "
                                          f"core ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
