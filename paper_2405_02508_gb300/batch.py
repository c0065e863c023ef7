"""Batched path: many items (a mesh seen by one camera) of uneven sizes in one launch per stage.

``BatchRenderer`` concatenates the meshes, plans the item table (``mer_batch_plan``)
and chains the batched C-ABI calls.  The raster and the backward are persistent
kernels that pull tiles of every item from a device work queue, so a step costs
the same handful of launches whatever the number of items; ``capture()`` records
the whole forward+backward step in one CUDA graph.

``PlainRenderer`` is the comparison path: one multi-stage launch sequence per item.

``autotune_tile`` times the bin tile sizes on the actual workload and caches the
winner per workload signature.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import binding as B
from .render import Renderer


class BatchRenderer:
    def __init__(self, meshes, items, cams, shading, C_attr: int, tex=None, tile: int = 32, persistent_ctas: int = 0,
                 device: str = "cuda", cover_hint: bool = True, precise: bool = False):
        """meshes: list of (verts [V,3] float32, tris [T,3] int32); items: list of (mesh, cam, H, W);
        cams: structured camera array; tex: texture tensor on the device or None.  cover_hint: the raster also
        writes the cover image and the backward skips the pixel pairs it shows cannot scatter (same results)."""
        self.device = device
        self.shading = shading
        self.C = shading.C
        self.C_attr = C_attr
        self.tile = tile
        self.persistent_ctas = persistent_ctas
        vo, to = [0], [0]
        for v, t in meshes:
            vo.append(vo[-1] + len(v))
            to.append(to[-1] + len(t))
        self.mesh_vert_off = vo
        self.n_verts = vo[-1]
        tris = np.concatenate([np.asarray(t, np.int32) for _, t in meshes]) if meshes else np.zeros((0, 3), np.int32)
        self.tris = torch.from_numpy(np.ascontiguousarray(tris)).to(device)
        arr = (B.MerItem * len(items))()
        for k, (mesh, cam, H, W) in enumerate(items):
            v, t = meshes[mesh]
            arr[k].V, arr[k].T, arr[k].H, arr[k].W = len(v), len(t), int(H), int(W)
            arr[k].cam = int(cam)
            arr[k].vert, arr[k].tri = vo[mesh], to[mesh]
        self.items_host = arr
        self.tot = B.mer_batch_plan(arr, tile)
        raw = np.frombuffer(bytes(arr), dtype=np.uint8).copy()
        self.items = torch.from_numpy(raw).to(device)
        self.item_pix = [(arr[k].pix, arr[k].H, arr[k].W) for k in range(len(items))]
        self.cams = B.cameras_tensor(cams, device)
        self.sh = B.shading_struct(shading, C_attr, tex, precise)
        self.bg = shading.bg_array()
        tot = self.tot
        self.vpix = torch.empty((max(tot.vrecs, 1), B.VERTEX_FLOATS), dtype=torch.float32, device=device)
        self.index = torch.empty(max(tot.pixels, 1), dtype=torch.int32, device=device)
        self.image = torch.empty((max(tot.pixels, 1), self.C), dtype=torch.float32, device=device)
        self.cover = torch.empty(max(tot.pixels, 1), dtype=torch.uint8, device=device) if cover_hint else None
        self.grad_vpix = torch.zeros((max(tot.vrecs, 1), 3), dtype=torch.float64, device=device)
        self.grad_verts = torch.zeros((max(self.n_verts, 1), 3), dtype=torch.float32, device=device)
        self._alloc_workspace(0)
        self.graph = None

    def _alloc_workspace(self, capacity: int, at_least: int = 0):
        nbytes = max(B.mer_batch_workspace_size(self.tot, capacity), at_least)
        self.workspace = torch.zeros((nbytes + 255) // 256 * 64, dtype=torch.float32, device=self.device)

    def ensure_backward_workspace(self, terms: int, grad_attr=None):
        """Grow the workspace to what a backward with these terms needs (MER_DETERMINISTIC keeps its fixed-point
        sums there); call before capturing a graph."""
        need = max(B.mer_backward_workspace_size(self.tot.vrecs, self.tot.mesh_rows,
                                                 B.attr_grad_channels(self.sh, grad_attr), terms),
                   B.mer_backward_workspace_size(self.tot.mesh_rows, 0, 0, terms))
        if self.workspace.numel() * 4 < need:
            self._alloc_workspace(0, need)
            self.graph = None

    # -- stages ------------------------------------------------------------------------------------
    def forward(self, verts, attr, tex=None, depth=None, bary=None, fused: bool = True):
        """Project, bin, raster and shade every item.  fused: raster and shade in one persistent pass
        (mer_batch_render); otherwise mer_batch_rasterize then mer_batch_shade (same results)."""
        B.mer_batch_project(verts, self.cams, self.items, self.tot, self.vpix)
        if fused:
            B.mer_batch_render(self.vpix, self.tris, self.items, self.tot, self.workspace, self.index, attr, tex,
                               self.bg, self.sh, self.image, depth, bary, self.persistent_ctas, self.cover)
            return self.image
        B.mer_batch_rasterize(self.vpix, self.tris, self.items, self.tot, self.workspace, self.index, depth, bary,
                              self.persistent_ctas, self.cover)
        B.mer_batch_shade(self.vpix, self.tris, self.items, self.tot, self.index, attr, tex, self.bg, self.sh,
                          self.image, self.workspace)
        return self.image

    def backward(self, grad_image, attr, tex=None, terms: int = 7, grad_attr=None):
        self.grad_vpix.zero_()
        self.grad_verts.zero_()
        if terms & B.MER_DETERMINISTIC:
            self.ensure_backward_workspace(terms, grad_attr)
        B.mer_batch_backward(self.vpix, self.tris, self.items, self.tot, self.index, self.image, grad_image, attr, tex,
                             self.sh, terms, self.grad_vpix, grad_attr, self.workspace, self.persistent_ctas,
                             self.cover)
        B.mer_batch_project_backward(self.cams, self.items, self.tot, self.vpix, self.grad_vpix, self.grad_verts,
                                     self.workspace if terms & B.MER_DETERMINISTIC else None)
        return self.grad_verts

    def step(self, verts, attr, grad_image, tex=None, terms: int = 7):
        self.forward(verts, attr, tex)
        return self.backward(grad_image, attr, tex, terms)

    def check(self):
        """Synchronise and raise if the device reported an overflow or an out-of-range index; on a bin
        overflow, resize the workspace to the exact need (the caller then reruns the step)."""
        code, total = B.mer_sync_status(self.workspace)
        if code == B.MER_EOVERFLOW:
            self._alloc_workspace(int(total * 1.25) + 1024)
            self.graph = None
        if code != B.MER_OK:
            raise B.MerError(code, "batched step")

    def prepare(self, verts, attr, tex=None):
        """One checked forward that sizes the bin lists exactly (before capturing a graph)."""
        self.forward(verts, attr, tex)
        try:
            self.check()
        except B.MerError as e:
            if e.code != B.MER_EOVERFLOW:
                raise
            self.forward(verts, attr, tex)
            self.check()

    # -- CUDA graph --------------------------------------------------------------------------------
    def capture(self, verts, attr, grad_image, tex=None, terms: int = 7):
        """Record one whole step (forward + backward) in a CUDA graph; replay with ``replay()``."""
        if self.persistent_ctas == 0:
            self.persistent_ctas = default_persistent_ctas()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):  # warm-up on the side stream, as graph capture requires
            self.step(verts, attr, grad_image, tex, terms)
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step(verts, attr, grad_image, tex, terms)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    # -- per item views ----------------------------------------------------------------------------
    def item_index(self, k):
        p, H, W = self.item_pix[k]
        return self.index[p:p + H * W].view(H, W)

    def item_image(self, k):
        p, H, W = self.item_pix[k]
        return self.image[p:p + H * W].view(H, W, self.C)

    def item_grad_vpix(self, k):
        it = self.items_host[k]
        return self.grad_vpix[it.vrec:it.vrec + it.V]


class PlainRenderer:
    """Comparison path: each item rendered by its own multi-stage launch sequence."""

    def __init__(self, meshes, items, cams, shading, C_attr: int, tex_shape=None, tile: int = 32,
                 device: str = "cuda", cover_hint: bool = True):
        self.meshes = meshes
        self.items = items
        self.cams = [B.cameras_tensor(cams[c:c + 1], device) for (_, c, _, _) in items]
        self.r = [Renderer(torch.from_numpy(np.asarray(meshes[m][1], np.int32)), len(meshes[m][0]), 1, H, W, shading,
                           C_attr, tex_shape, tile, device, cover_hint) for (m, _, H, W) in items]

    def step(self, verts_list, attr_list, grads, tex=None, checked=False):
        out = []
        for k, (m, _, _, _) in enumerate(self.items):
            r = self.r[k]
            r.forward(verts_list[m], self.cams[k], attr_list[m], tex, checked=checked)
            out.append(r.backward(grads[k], self.cams[k], attr_list[m], tex))
        return out


def default_persistent_ctas() -> int:
    """Persistent grid: the number of raster CTAs that fit on the device at once (4 per SM; the backward
    scales it to its own 6 per SM)."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    return int(props.multi_processor_count) * 4


_CACHE_FILE = os.path.join(os.path.expanduser("~"), ".cache", "mer_autotune.json")


def autotune_tile(make_renderer, run_step, candidates=(16, 32, 64), reps: int = 3, key: str | None = None,
                  cache_file: str | None = _CACHE_FILE) -> tuple[int, dict]:
    """Time one step per candidate bin tile size and return (best tile, {tile: ms}).

    make_renderer(tile) builds a renderer; run_step(renderer) runs one step on the current stream.
    The result is cached under ``key`` (a workload signature) in memory and in ``cache_file``."""
    cache = {}
    if key and cache_file and os.path.exists(cache_file):
        try:
            with open(cache_file) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key and key in cache:
        return int(cache[key]["tile"]), cache[key]["ms"]
    times = {}
    for tile in candidates:
        r = make_renderer(tile)
        run_step(r)  # warm-up (sizes the workspace)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run_step(r)
        e1.record()
        torch.cuda.synchronize()
        times[tile] = e0.elapsed_time(e1) / reps
        del r
    best = min(times, key=times.get)
    if key and cache_file:
        cache[key] = {"tile": best, "ms": {str(k): v for k, v in times.items()}}
        try:
            os.makedirs(os.path.dirname(cache_file), exist_ok=True)
            with open(cache_file, "w") as f:
                json.dump(cache, f)
        except OSError:
            pass
    return best, times


def autotune(make_renderer, run_step, tiles=(16, 32, 64), ctas_per_sm=(1, 2, 4), reps: int = 3, key: str | None = None,
             cache_file: str | None = _CACHE_FILE) -> tuple[int, int, dict]:
    """Bin tile size and work split (persistent CTAs of the raster and backward grids) by timing one step per
    candidate pair -> (tile, persistent CTAs, {"tile/ctas": ms}).  make_renderer(tile, ctas) builds a
    renderer; the result is cached under ``key`` like autotune_tile's."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    cache = {}
    if key and cache_file and os.path.exists(cache_file):
        try:
            with open(cache_file) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    ckey = None if key is None else key + "_split"
    if ckey and ckey in cache:
        return int(cache[ckey]["tile"]), int(cache[ckey]["ctas"]), cache[ckey]["ms"]
    times = {}
    for tile in tiles:
        for c in ctas_per_sm:
            r = make_renderer(tile, sms * c)
            run_step(r)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                run_step(r)
            e1.record()
            torch.cuda.synchronize()
            times[f"{tile}/{sms * c}"] = e0.elapsed_time(e1) / reps
            del r
    best = min(times, key=times.get)
    tile, ctas = (int(v) for v in best.split("/"))
    if ckey and cache_file:
        cache[ckey] = {"tile": tile, "ctas": ctas, "ms": times}
        try:
            os.makedirs(os.path.dirname(cache_file), exist_ok=True)
            with open(cache_file, "w") as f:
                json.dump(cache, f)
        except OSError:
            pass
    return tile, ctas, times


def workload_key(items, meshes) -> str:
    """Autotune signature: triangle and pixel totals rounded to powers of two."""
    T = sum(len(meshes[m][1]) for (m, _, _, _) in items)
    P = sum(H * W for (_, _, H, W) in items)
    return f"T{int(np.log2(max(T, 1)))}_P{int(np.log2(max(P, 1)))}_n{len(items)}"
