"""GB300 light-field-probe ray tracer (Liu, Nowrouzezahrai & McGuire, arXiv 2507.14624).

``lfp`` is the ctypes binding of the C ABI (include/lfp.h). This module adds a
thin torch-facing layer: device buffers are torch tensors, streams are torch
streams, and ``render`` is differentiable with respect to probe radiance
through the hand-written adjoint kernel. Nothing here computes any step of the
tracer; it only allocates, marshals arguments and calls the library.
"""
from __future__ import annotations

import ctypes

from . import lfp
from .lfp import (LFP_CLASS_HIT, LFP_CLASS_MISS, LFP_CLASS_STEPLIMIT, LFP_CLASS_UNKNOWN, LFP_ENGINE_NESTED,
                  LFP_ENGINE_STREAM, LFP_MARCH_FLAT, LFP_MARCH_HIER, LFP_SCHED_PERSISTENT, LFP_SCHED_TILES,
                  LFP_TEXEL_F16, LFP_TEXEL_F32, LfpError)

__all__ = ["lfp", "ProbeGrid", "ProbeHierarchy", "make_views", "render", "render_levels", "LfpError", "LFP_TEXEL_F32", "LFP_TEXEL_F16",
           "LFP_CLASS_MISS", "LFP_CLASS_HIT", "LFP_CLASS_UNKNOWN", "LFP_CLASS_STEPLIMIT",
           "LFP_MARCH_HIER", "LFP_MARCH_FLAT", "LFP_SCHED_TILES", "LFP_SCHED_PERSISTENT", "LFP_ENGINE_STREAM",
           "LFP_ENGINE_NESTED"]


def _stream_handle(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def make_views(views) -> tuple:
    """Pack camera views (objects with pos, right, up, fwd, fov_y, W, H) into a
    ctypes lfp_view array with consecutive output offsets. Returns
    (array, n_views, total_pixels)."""
    arr = (lfp.lfp_view * len(views))()
    off = 0
    for k, v in enumerate(views):
        a = arr[k]
        for i in range(3):
            a.pos[i], a.right[i], a.up[i], a.fwd[i] = v.pos[i], v.right[i], v.up[i], v.fwd[i]
        a.fov_y, a.W, a.H, a.out_offset = v.fov_y, v.W, v.H, off
        off += v.W * v.H
    return arr, len(views), off


_LIB_DIGEST = None


def _library_digest() -> str:
    """sha256 of the loaded CUDA library (a rebuild invalidates tuned picks)."""
    global _LIB_DIGEST
    if _LIB_DIGEST is None:
        import hashlib
        with open(lfp.LIB_PATH, "rb") as f:
            _LIB_DIGEST = hashlib.sha256(f.read()).hexdigest()[:16]
    return _LIB_DIGEST


def tune_key(grid, views, device_name: str | None = None) -> str:
    """Key of an autotuner pick: GPU, library build, grid descriptor and the
    multiset of view sizes (the views' poses do not enter)."""
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    d = grid.desc
    desc = (d.nx, d.ny, d.nz, d.spacing, d.N, d.M, d.radiance_fmt, d.normal_fmt, d.thickness_rel, d.max_steps,
            d.eye_lookup, d.traversal)
    sizes = sorted((v.W, v.H) for v in views)
    return f"{device_name}|{_library_digest()}|{desc}|{sizes}"


def _read_tune_cache(path: str) -> dict:
    import json
    import os
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def _write_tune_cache(path: str, key: str, pick: dict) -> None:
    import json
    import os
    data = _read_tune_cache(path)
    data[key] = {k: (list(v) if isinstance(v, tuple) else v) for k, v in pick.items()}
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class ProbeGrid:
    """A probe grid on the current CUDA device (owns one lfp_grid handle).

    spec: object with nx, ny, nz, origin, spacing, N, M (e.g. synth.Grid).
    eye_lookup: lfp.LFP_EYE_BILINEAR / LFP_EYE_NEAREST; traversal:
    lfp.LFP_TRAVERSAL_GRID / LFP_TRAVERSAL_NEAREST (at most 8 probes).
    """

    def __init__(self, spec, radiance_fmt=LFP_TEXEL_F32, normal_fmt=LFP_TEXEL_F32, thickness_rel=1.0,
                 eye_eps=0.0, max_steps=0, eye_lookup=0, traversal=0):
        d = lfp.lfp_grid_desc()
        d.nx, d.ny, d.nz = spec.nx, spec.ny, spec.nz
        for i in range(3):
            d.origin[i] = spec.origin[i]
        d.spacing, d.N, d.M = spec.spacing, spec.N, spec.M
        d.radiance_fmt, d.normal_fmt = radiance_fmt, normal_fmt
        d.thickness_rel, d.eye_eps, d.max_steps = thickness_rel, eye_eps, max_steps
        d.eye_lookup, d.traversal = eye_lookup, traversal
        self.desc = d
        self.spec = spec
        self.N, self.M = spec.N, spec.M
        self.n_probes = spec.nx * spec.ny * spec.nz
        self.handle = lfp.lfp_create_grid(d)

    def close(self):
        if getattr(self, "handle", None):
            lfp.lfp_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def device_bytes(self) -> int:
        return lfp.lfp_grid_bytes(self.desc)

    @property
    def skip_blocks(self) -> list:
        """Block sides of the grid's skip levels (lfp_skip_blocks), ascending."""
        return lfp.lfp_skip_blocks(self.desc)

    def upload(self, dist, normal, radiance, first_probe=0, stream=None):
        """Upload probe maps (numpy float32 host arrays or CUDA float32 tensors):
        dist [P][N][N], normal [P][N][N][3], radiance [P][N][N][3]."""
        import numpy as np
        import torch
        pl = lfp.lfp_probe_planes()
        if isinstance(dist, torch.Tensor):
            keep = [t.contiguous() for t in (dist, normal, radiance)]
            for t in keep:
                if t.dtype != torch.float32 or not t.is_cuda:
                    raise ValueError("device probe planes must be CUDA float32 tensors")
            pl.dist, pl.normal, pl.radiance = (t.data_ptr() for t in keep)
            pl.is_device = 1
        else:
            keep = [np.ascontiguousarray(a, dtype=np.float32) for a in (dist, normal, radiance)]
            pl.dist, pl.normal, pl.radiance = (a.ctypes.data for a in keep)
            pl.is_device = 0
        count = keep[0].shape[0]
        s = _stream_handle(stream)
        lfp.lfp_upload_probes(self.handle, first_probe, count, pl, s)
        if not pl.is_device:  # host planes must outlive the asynchronous copies
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def build_from_points(self, xyz, rgb, normal=None, first_probe=0, count=None, empty_dist=0.0, stream=None):
        """Fill probes [first_probe, first_probe + count) from a point cloud
        (lfp_build_probes_from_points): xyz, rgb, optional normal [n][3]
        float32: CUDA tensors (read in place), or numpy arrays / CPU tensors
        (copied; pinned CPU tensors copy asynchronously)."""
        import numpy as np
        import torch
        count = self.n_probes - first_probe if count is None else count
        pc = lfp.lfp_point_cloud()
        arrays = [xyz, rgb] + ([normal] if normal is not None else [])
        if isinstance(xyz, torch.Tensor):
            keep = [t.contiguous() for t in arrays]
            for t in keep:
                if t.dtype != torch.float32 or t.is_cuda != keep[0].is_cuda:
                    raise ValueError("point clouds must be float32 tensors on one device")
            ptr = [t.data_ptr() for t in keep]
            pc.is_device = 1 if keep[0].is_cuda else 0
        else:
            keep = [np.ascontiguousarray(a, dtype=np.float32) for a in arrays]
            ptr = [a.ctypes.data for a in keep]
            pc.is_device = 0
        pc.xyz, pc.rgb = ptr[0], ptr[1]
        pc.normal = ptr[2] if normal is not None else None
        pc.n = keep[0].shape[0]
        lfp.lfp_build_probes_from_points(self.handle, first_probe, count, pc, empty_dist, _stream_handle(stream))
        if not pc.is_device:  # host planes must outlive the asynchronous copies
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def read_probes(self, first_probe=0, count=None, stream=None):
        """(dist [c][N][N], normal [c][N][N][3], radiance [c][N][N][3]) float32 CUDA tensors."""
        import torch
        count = self.n_probes - first_probe if count is None else count
        dev = torch.device("cuda", torch.cuda.current_device())
        d = torch.empty((count, self.N, self.N), dtype=torch.float32, device=dev)
        n = torch.empty((count, self.N, self.N, 3), dtype=torch.float32, device=dev)
        r = torch.empty((count, self.N, self.N, 3), dtype=torch.float32, device=dev)
        lfp.lfp_read_probes(self.handle, first_probe, count, ctypes.c_void_p(d.data_ptr()),
                            ctypes.c_void_p(n.data_ptr()), ctypes.c_void_p(r.data_ptr()), _stream_handle(stream))
        return d, n, r

    def set_radiance(self, radiance, stream=None):
        """Replace all probes' radiance from a CUDA float32 tensor [P][N][N][3]."""
        r = radiance.contiguous()
        lfp.lfp_set_radiance(self.handle, ctypes.c_void_p(r.data_ptr()), _stream_handle(stream))

    def render(self, views, aux=True, hit_texel=False, counters=False, march=LFP_MARCH_HIER, tile=None,
               schedule=0, engine=0, occupancy=0, skip_block=0, stream=None):
        """Render views; returns a dict of CUDA tensors: rgb [P,3] f32,
        cls [P] u8, and optionally probe [P] i32, uv [P,2] f32, texel [P] i32,
        counters [8] i64 (see lfp.COUNTER_NAMES). skip_block: one of
        skip_blocks, 0 for the grid's default."""
        import torch
        arr, n, total = make_views(views)
        dev = torch.device("cuda", torch.cuda.current_device())
        out = {"rgb": torch.empty((total, 3), dtype=torch.float32, device=dev),
               "cls": torch.empty(total, dtype=torch.uint8, device=dev)}
        if aux:
            out["probe"] = torch.empty(total, dtype=torch.int32, device=dev)
            out["uv"] = torch.empty((total, 2), dtype=torch.float32, device=dev)
        if hit_texel:
            out["texel"] = torch.empty(total, dtype=torch.int32, device=dev)
        if counters:
            out["counters"] = torch.zeros(lfp.N_COUNTERS, dtype=torch.int64, device=dev)
        o = lfp.lfp_outputs()
        o.rgb, o.cls = out["rgb"].data_ptr(), out["cls"].data_ptr()
        o.aux_probe = out["probe"].data_ptr() if aux else None
        o.aux_uv = out["uv"].data_ptr() if aux else None
        o.hit_texel = out["texel"].data_ptr() if hit_texel else None
        o.counters = out["counters"].data_ptr() if counters else None
        opts = lfp.lfp_render_opts()
        opts.march = march
        if tile is not None:
            opts.tile_w, opts.tile_h = tile
        opts.schedule = schedule
        opts.engine = engine
        opts.occupancy = occupancy
        opts.skip_block = skip_block
        lfp.lfp_render_ex(self.handle, arr, n, o, opts, _stream_handle(stream))
        return out

    def autotune(self, views, stream=None, cache: str | None = None) -> dict:
        """Pick the fastest launch configuration for these views (kept as the
        grid default). Returns it as a dict. With `cache` (a JSON file), a
        pick stored there for the same GPU, library build, grid and view
        sizes is applied without timing; a new pick is added to the file."""
        import torch
        key = tune_key(self, views) if cache else None
        if cache:
            got = _read_tune_cache(cache).get(key)
            if got is not None:
                opts = lfp.lfp_render_opts()
                opts.engine, opts.schedule, opts.occupancy = got["engine"], got["schedule"], got["occupancy"]
                opts.tile_w, opts.tile_h = got["tile"]
                opts.skip_block = got.get("skip_block", 0)
                lfp.lfp_set_defaults(self.handle, opts)
                return dict(got, tile=tuple(got["tile"]), cached=True)
        arr, n, total = make_views(views)
        dev = torch.device("cuda", torch.cuda.current_device())
        rgb = torch.empty((total, 3), dtype=torch.float32, device=dev)
        cls = torch.empty(total, dtype=torch.uint8, device=dev)
        o = lfp.lfp_outputs()
        o.rgb, o.cls = rgb.data_ptr(), cls.data_ptr()
        b = lfp.lfp_autotune(self.handle, arr, n, o, _stream_handle(stream))
        pick = {"engine": b.engine, "tile": (b.tile_w, b.tile_h), "schedule": b.schedule, "occupancy": b.occupancy,
                "skip_block": b.skip_block}
        if cache:
            _write_tune_cache(cache, key, pick)
        return pick

    def render_graph(self, views, aux=False, engine=0, occupancy=0, skip_block=0, stream=None):
        """Capture one render of these views in a CUDA graph (outputs are
        preallocated and reused). Returns (graph, outputs); graph.replay()
        re-renders into the same tensors. engine / occupancy / skip_block as
        in render (0: the grid's default)."""
        import torch
        s = torch.cuda.Stream() if stream is None else stream
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            out = self.render(views, aux=aux, engine=engine, occupancy=occupancy, skip_block=skip_block,
                              stream=s)  # warm-up outside capture
        torch.cuda.current_stream().wait_stream(s)
        arr, n, total = make_views(views)
        o = lfp.lfp_outputs()
        o.rgb, o.cls = out["rgb"].data_ptr(), out["cls"].data_ptr()
        o.aux_probe = out["probe"].data_ptr() if aux else None
        o.aux_uv = out["uv"].data_ptr() if aux else None
        opts = lfp.lfp_render_opts()
        opts.engine = engine
        opts.occupancy = occupancy
        opts.skip_block = skip_block
        graph = torch.cuda.CUDAGraph()
        keep = (arr, o, opts)
        with torch.cuda.graph(graph, stream=s):
            lfp.lfp_render_ex(self.handle, arr, n, o, opts, _stream_handle(s))
        graph._lfp_keep = keep
        return graph, out

    def render_backward(self, views, grad_rgb, cls, probe, uv, grad_radiance=None, reduction=0, stream=None):
        """Adjoint: accumulate into grad_radiance [P][N][N][3] f32 (zeros if None) and return it.
        reduction: lfp.LFP_REDUCE_* (atomics, warp-aggregated, sort by texel)."""
        import torch
        arr, n, total = make_views(views)
        if grad_radiance is None:
            grad_radiance = torch.zeros((self.n_probes, self.N, self.N, 3), dtype=torch.float32,
                                        device=grad_rgb.device)
        g = grad_rgb.contiguous()
        lfp.lfp_render_backward_ex(self.handle, arr, n, ctypes.c_void_p(g.data_ptr()),
                                   ctypes.c_void_p(cls.data_ptr()), ctypes.c_void_p(probe.data_ptr()),
                                   ctypes.c_void_p(uv.data_ptr()), ctypes.c_void_p(grad_radiance.data_ptr()),
                                   reduction, _stream_handle(stream))
        return grad_radiance

    def render_to_host(self, views, rgb_host, cls_host, stream=None):
        """One C-ABI call: render into grid-owned device buffers and copy rgb
        and cls into the given host tensors (pinned for asynchronous copies)."""
        arr, n, total = make_views(views)
        lfp.lfp_render_to_host(self.handle, arr, n, ctypes.c_void_p(rgb_host.data_ptr()),
                               ctypes.c_void_p(cls_host.data_ptr()), _stream_handle(stream))

    def render_to_host_async(self, views, rgb_host, cls_host, stream=None):
        """Queue a render whose rgb / cls land in the given pinned host tensors
        (lfp_render_to_host_async); they are complete after sync_host()."""
        arr, n, total = make_views(views)
        lfp.lfp_render_to_host_async(self.handle, arr, n, ctypes.c_void_p(rgb_host.data_ptr()),
                                     ctypes.c_void_p(cls_host.data_ptr()), _stream_handle(stream))

    def sync_host(self):
        lfp.lfp_sync_host(self.handle)

    def check_flags(self, stream=None) -> int:
        return lfp.lfp_check_flags(self.handle, _stream_handle(stream))


class ProbeHierarchy:
    """Multi-scale hierarchy: ProbeGrids of one scene at several spacings
    (see lfp_render_levels in include/lfp.h). Each view is traced in the
    finest level whose probe box holds its camera."""

    def __init__(self, grids):
        self.grids = list(grids)
        self.handles = [g.handle for g in self.grids]

    def level_of(self, views) -> list:
        arr, n, _ = make_views(views)
        return lfp.lfp_pick_levels(self.handles, arr, n)

    def _outputs(self, total, aux, hit_texel, counters):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        out = {"rgb": torch.empty((total, 3), dtype=torch.float32, device=dev),
               "cls": torch.empty(total, dtype=torch.uint8, device=dev)}
        if aux:
            out["probe"] = torch.empty(total, dtype=torch.int32, device=dev)
            out["uv"] = torch.empty((total, 2), dtype=torch.float32, device=dev)
        if hit_texel:
            out["texel"] = torch.empty(total, dtype=torch.int32, device=dev)
        if counters:
            out["counters"] = torch.zeros(lfp.N_COUNTERS, dtype=torch.int64, device=dev)
        o = lfp.lfp_outputs()
        o.rgb, o.cls = out["rgb"].data_ptr(), out["cls"].data_ptr()
        o.aux_probe = out["probe"].data_ptr() if aux else None
        o.aux_uv = out["uv"].data_ptr() if aux else None
        o.hit_texel = out["texel"].data_ptr() if hit_texel else None
        o.counters = out["counters"].data_ptr() if counters else None
        return out, o

    def autotune(self, views, stream=None) -> dict:
        """Pick each level's launch configuration and skip level on the views
        that level renders (ProbeGrid.autotune per level); returns {level: pick}."""
        lev = self.level_of(views)
        picks = {}
        for k, g in enumerate(self.grids):
            mine = [v for v, l in zip(views, lev) if l == k]
            if mine:
                picks[k] = g.autotune(mine, stream=stream)
        return picks

    def render(self, views, aux=True, hit_texel=False, counters=False, engine=0, occupancy=0, skip_block=0,
               stream=None):
        """Like ProbeGrid.render; `probe` indexes the probes of each view's
        level. A nonzero skip_block must be a skip level of every level that
        renders a view (0: each level's default)."""
        arr, n, total = make_views(views)
        out, o = self._outputs(total, aux, hit_texel, counters)
        opts = lfp.lfp_render_opts()
        opts.engine = engine
        opts.occupancy = occupancy
        opts.skip_block = skip_block
        lfp.lfp_render_levels(self.handles, arr, n, o, opts, _stream_handle(stream))
        return out

    def render_graph(self, views, aux=False, engine=0, occupancy=0, skip_block=0, stream=None):
        """One hierarchy render captured in a CUDA graph (outputs reused);
        engine / occupancy / skip_block as in render (0: each level's default)."""
        import torch
        s = torch.cuda.Stream() if stream is None else stream
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            out = self.render(views, aux=aux, engine=engine, occupancy=occupancy, skip_block=skip_block, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        arr, n, total = make_views(views)
        o = lfp.lfp_outputs()
        o.rgb, o.cls = out["rgb"].data_ptr(), out["cls"].data_ptr()
        o.aux_probe = out["probe"].data_ptr() if aux else None
        o.aux_uv = out["uv"].data_ptr() if aux else None
        opts = lfp.lfp_render_opts()
        opts.engine = engine
        opts.occupancy = occupancy
        opts.skip_block = skip_block
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            lfp.lfp_render_levels(self.handles, arr, n, o, opts, _stream_handle(s))
        graph._lfp_keep = (arr, o, opts)
        return graph, out

    def render_backward(self, views, grad_rgb, cls, probe, uv, grads=None, reduction=0, stream=None):
        """Adjoint into one [P][N][N][3] f32 accumulator per level (zeros if
        None); returns the list."""
        import torch
        arr, n, total = make_views(views)
        if grads is None:
            grads = [torch.zeros((g.n_probes, g.N, g.N, 3), dtype=torch.float32, device=grad_rgb.device)
                     for g in self.grids]
        gr = grad_rgb.contiguous()
        lfp.lfp_render_backward_levels(self.handles, arr, n, ctypes.c_void_p(gr.data_ptr()),
                                       ctypes.c_void_p(cls.data_ptr()), ctypes.c_void_p(probe.data_ptr()),
                                       ctypes.c_void_p(uv.data_ptr()), [t.data_ptr() for t in grads], reduction,
                                       _stream_handle(stream))
        return grads


def _autograd():
    import torch

    class LfpRender(torch.autograd.Function):
        """rgb = render(radiance): forward through the tracer, backward through
        the adjoint kernel (rgb is linear in radiance for fixed geometry)."""

        @staticmethod
        def forward(ctx, radiance, grid: ProbeGrid, views):
            grid.set_radiance(radiance.detach())
            out = grid.render(views, aux=True)
            ctx.grid, ctx.views = grid, views
            ctx.save_for_backward(out["cls"], out["probe"], out["uv"])
            ctx.mark_non_differentiable(out["cls"])
            return out["rgb"], out["cls"]

        @staticmethod
        def backward(ctx, grad_rgb, grad_cls):
            cls, probe, uv = ctx.saved_tensors
            g = ctx.grid.render_backward(ctx.views, grad_rgb, cls, probe, uv)
            return g, None, None

    class LfpRenderLevels(torch.autograd.Function):
        """rgb = render over a hierarchy of the per-level radiance tensors."""

        @staticmethod
        def forward(ctx, hierarchy, views, *radiances):
            for g, r in zip(hierarchy.grids, radiances):
                g.set_radiance(r.detach())
            out = hierarchy.render(views, aux=True)
            ctx.hierarchy, ctx.views = hierarchy, views
            ctx.save_for_backward(out["cls"], out["probe"], out["uv"])
            ctx.mark_non_differentiable(out["cls"])
            return out["rgb"], out["cls"]

        @staticmethod
        def backward(ctx, grad_rgb, grad_cls):
            cls, probe, uv = ctx.saved_tensors
            grads = ctx.hierarchy.render_backward(ctx.views, grad_rgb, cls, probe, uv)
            return (None, None, *grads)

    return LfpRender, LfpRenderLevels


_LfpRender = None
_LfpRenderLevels = None


def render(radiance, grid: ProbeGrid, views):
    """Differentiable render: radiance [P][N][N][3] f32 CUDA tensor -> (rgb [pixels,3], cls [pixels])."""
    global _LfpRender, _LfpRenderLevels
    if _LfpRender is None:
        _LfpRender, _LfpRenderLevels = _autograd()
    return _LfpRender.apply(radiance, grid, views)


def render_levels(radiances, hierarchy: ProbeHierarchy, views):
    """Differentiable hierarchy render: one radiance tensor [P_l][N_l][N_l][3]
    per level -> (rgb [pixels,3], cls [pixels])."""
    global _LfpRender, _LfpRenderLevels
    if _LfpRender is None:
        _LfpRender, _LfpRenderLevels = _autograd()
    return _LfpRenderLevels.apply(hierarchy, views, *radiances)
