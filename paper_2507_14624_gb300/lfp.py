"""ctypes binding of the C ABI in include/lfp.h (argument marshalling only).

Every function here has the name of the C entry point it calls; every step of
the tracer runs in the CUDA library. PyTorch supplies device memory (tensor
data pointers) and streams. The library is loaded from the package directory
(liblfp.so, or with LFP_CHECKED=1 the checked build liblfp_checked.so); if it
is missing the import fails -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblfp_checked.so" if os.environ.get("LFP_CHECKED") == "1" else "liblfp.so")

# status codes
LFP_OK, LFP_ERR_INVALID_ARG, LFP_ERR_OOM, LFP_ERR_CUDA, LFP_ERR_STATE, LFP_ERR_CAPACITY = 0, 1, 2, 3, 4, 5
LFP_ERR_BOUNDS = 6
LFP_STATIC_MAX_VIEWS = 4096
LFP_WARN_STEPLIMIT = 100
LFP_TEXEL_F32, LFP_TEXEL_F16 = 0, 1
LFP_CLASS_MISS, LFP_CLASS_HIT, LFP_CLASS_UNKNOWN, LFP_CLASS_STEPLIMIT = 0, 1, 2, 3
LFP_MARCH_HIER, LFP_MARCH_FLAT = 0, 1
LFP_SCHED_AUTO, LFP_SCHED_TILES, LFP_SCHED_PERSISTENT = 0, 1, 2
LFP_ENGINE_AUTO, LFP_ENGINE_STREAM, LFP_ENGINE_NESTED = 0, 1, 2
LFP_REDUCE_AUTO, LFP_REDUCE_ATOMIC, LFP_REDUCE_WARP, LFP_REDUCE_SORT = 0, 1, 2, 3
LFP_OCC_AUTO, LFP_OCC_8, LFP_OCC_9 = 0, 1, 2
LFP_EYE_BILINEAR, LFP_EYE_NEAREST = 0, 1
LFP_TRAVERSAL_GRID, LFP_TRAVERSAL_NEAREST = 0, 1
LFP_NEAREST_MAX_PROBES = 8
LFP_MAX_SKIP_LEVELS = 4
N_COUNTERS = 8
COUNTER_NAMES = ("coarse", "fine", "normal", "radiance", "cells", "probes", "hits", "rays")


class lfp_grid_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("origin", ctypes.c_float * 3), ("spacing", ctypes.c_float),
                ("N", ctypes.c_int), ("M", ctypes.c_int),
                ("radiance_fmt", ctypes.c_int), ("normal_fmt", ctypes.c_int),
                ("thickness_rel", ctypes.c_float), ("eye_eps", ctypes.c_float),
                ("max_steps", ctypes.c_int), ("eye_lookup", ctypes.c_int), ("traversal", ctypes.c_int)]


class lfp_view(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_float * 3), ("right", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("fwd", ctypes.c_float * 3), ("fov_y", ctypes.c_float), ("W", ctypes.c_int),
                ("H", ctypes.c_int), ("out_offset", ctypes.c_longlong)]


class lfp_probe_planes(ctypes.Structure):
    _fields_ = [("dist", ctypes.c_void_p), ("normal", ctypes.c_void_p), ("radiance", ctypes.c_void_p),
                ("is_device", ctypes.c_int)]


class lfp_outputs(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("cls", ctypes.c_void_p), ("aux_probe", ctypes.c_void_p),
                ("aux_uv", ctypes.c_void_p), ("hit_texel", ctypes.c_void_p), ("counters", ctypes.c_void_p)]


class lfp_render_opts(ctypes.Structure):
    _fields_ = [("march", ctypes.c_int), ("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int),
                ("schedule", ctypes.c_int), ("engine", ctypes.c_int), ("occupancy", ctypes.c_int),
                ("skip_block", ctypes.c_int)]


class lfp_point_cloud(ctypes.Structure):
    _fields_ = [("xyz", ctypes.c_void_p), ("rgb", ctypes.c_void_p), ("normal", ctypes.c_void_p),
                ("n", ctypes.c_longlong), ("is_device", ctypes.c_int)]


class LfpError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {lfp_status_string(status)} ({status})")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is missing: run paper_2507_14624_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, P = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER
    sig = {
        "lfp_create_grid": ([P(lfp_grid_desc), P(vp)], i),
        "lfp_upload_probes": ([vp, i, i, P(lfp_probe_planes), vp], i),
        "lfp_render": ([vp, P(lfp_view), i, vp, vp, vp, vp, vp], i),
        "lfp_render_ex": ([vp, P(lfp_view), i, P(lfp_outputs), P(lfp_render_opts), vp], i),
        "lfp_render_to_host": ([vp, P(lfp_view), i, vp, vp, vp], i),
        "lfp_render_to_host_async": ([vp, P(lfp_view), i, vp, vp, vp], i),
        "lfp_sync_host": ([vp], i),
        "lfp_render_static": ([vp, P(lfp_view), i, P(lfp_outputs), vp], i),
        "lfp_autotune": ([vp, P(lfp_view), i, P(lfp_outputs), P(lfp_render_opts), vp], i),
        "lfp_set_defaults": ([vp, P(lfp_render_opts)], i),
        "lfp_render_backward": ([vp, P(lfp_view), i, vp, vp, vp, vp, vp, vp], i),
        "lfp_render_backward_ex": ([vp, P(lfp_view), i, vp, vp, vp, vp, vp, i, vp], i),
        "lfp_build_probes_from_points": ([vp, i, i, P(lfp_point_cloud), ctypes.c_float, vp], i),
        "lfp_read_probes": ([vp, i, i, vp, vp, vp, vp], i),
        "lfp_pick_levels": ([P(vp), i, P(lfp_view), i, P(ctypes.c_int32)], i),
        "lfp_render_levels": ([P(vp), i, P(lfp_view), i, P(lfp_outputs), P(lfp_render_opts), vp], i),
        "lfp_render_backward_levels": ([P(vp), i, P(lfp_view), i, vp, vp, vp, vp, P(vp), i, vp], i),
        "lfp_set_radiance": ([vp, vp, vp], i),
        "lfp_check_flags": ([vp, vp], i),
        "lfp_grid_bytes": ([P(lfp_grid_desc), P(ctypes.c_ulonglong)], i),
        "lfp_skip_blocks": ([P(lfp_grid_desc), P(i), P(i)], i),
        "lfp_destroy_grid": ([vp], None),
        "lfp_status_string": ([i], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def _check(status: int, what: str) -> int:
    if status not in (LFP_OK, LFP_WARN_STEPLIMIT):
        raise LfpError(status, what)
    return status


def lfp_status_string(status: int) -> str:
    return _lib.lfp_status_string(status).decode()


def lfp_create_grid(desc: lfp_grid_desc) -> int:
    h = ctypes.c_void_p()
    _check(_lib.lfp_create_grid(ctypes.byref(desc), ctypes.byref(h)), "lfp_create_grid")
    return h.value


def lfp_destroy_grid(grid) -> None:
    _lib.lfp_destroy_grid(grid)


def lfp_upload_probes(grid, first_probe: int, count: int, planes: lfp_probe_planes, stream) -> None:
    _check(_lib.lfp_upload_probes(grid, first_probe, count, ctypes.byref(planes), stream), "lfp_upload_probes")


def lfp_render(grid, views, n_views, rgb, cls, aux_probe, aux_uv, stream) -> None:
    _check(_lib.lfp_render(grid, views, n_views, rgb, cls, aux_probe, aux_uv, stream), "lfp_render")


def lfp_render_ex(grid, views, n_views, outputs: lfp_outputs, opts: lfp_render_opts | None, stream) -> None:
    _check(_lib.lfp_render_ex(grid, views, n_views, ctypes.byref(outputs),
                              ctypes.byref(opts) if opts is not None else None, stream), "lfp_render_ex")


def lfp_render_static(grid, views, n_views, outputs: lfp_outputs, stream) -> None:
    """Forward render that allocates nothing (fixed scratch; see include/lfp.h)."""
    _check(_lib.lfp_render_static(grid, views, n_views, ctypes.byref(outputs), stream), "lfp_render_static")


def lfp_autotune(grid, views, n_views, outputs: lfp_outputs, stream) -> lfp_render_opts:
    """Time the launch configurations, keep the fastest as the grid default, return it."""
    best = lfp_render_opts()
    _check(_lib.lfp_autotune(grid, views, n_views, ctypes.byref(outputs), ctypes.byref(best), stream), "lfp_autotune")
    return best


def lfp_set_defaults(grid, opts: lfp_render_opts) -> None:
    """Make opts the grid's default launch configuration."""
    _check(_lib.lfp_set_defaults(grid, ctypes.byref(opts)), "lfp_set_defaults")


def lfp_render_to_host(grid, views, n_views, rgb_host, cls_host, stream) -> None:
    _check(_lib.lfp_render_to_host(grid, views, n_views, rgb_host, cls_host, stream), "lfp_render_to_host")


def lfp_render_to_host_async(grid, views, n_views, rgb_host, cls_host, stream) -> None:
    _check(_lib.lfp_render_to_host_async(grid, views, n_views, rgb_host, cls_host, stream), "lfp_render_to_host_async")


def lfp_sync_host(grid) -> None:
    _check(_lib.lfp_sync_host(grid), "lfp_sync_host")


def lfp_render_backward(grid, views, n_views, grad_rgb, cls, aux_probe, aux_uv, grad_radiance, stream) -> None:
    _check(_lib.lfp_render_backward(grid, views, n_views, grad_rgb, cls, aux_probe, aux_uv, grad_radiance, stream),
           "lfp_render_backward")


def lfp_render_backward_ex(grid, views, n_views, grad_rgb, cls, aux_probe, aux_uv, grad_radiance, reduction,
                           stream) -> None:
    _check(_lib.lfp_render_backward_ex(grid, views, n_views, grad_rgb, cls, aux_probe, aux_uv, grad_radiance,
                                       reduction, stream), "lfp_render_backward_ex")


def lfp_build_probes_from_points(grid, first_probe, count, cloud: lfp_point_cloud, empty_dist, stream) -> None:
    _check(_lib.lfp_build_probes_from_points(grid, first_probe, count, ctypes.byref(cloud), empty_dist, stream),
           "lfp_build_probes_from_points")


def lfp_read_probes(grid, first_probe, count, dist, normal, radiance, stream) -> None:
    _check(_lib.lfp_read_probes(grid, first_probe, count, dist, normal, radiance, stream), "lfp_read_probes")


def _handles(grids):
    arr = (ctypes.c_void_p * len(grids))()
    for k, g in enumerate(grids):
        arr[k] = g
    return arr


def lfp_pick_levels(levels, views, n_views) -> list:
    """Level that traces each view in a multi-scale hierarchy (see include/lfp.h)."""
    out = (ctypes.c_int32 * n_views)()
    _check(_lib.lfp_pick_levels(_handles(levels), len(levels), views, n_views, out), "lfp_pick_levels")
    return list(out)


def lfp_render_levels(levels, views, n_views, outputs: lfp_outputs, opts: lfp_render_opts | None, stream) -> None:
    _check(_lib.lfp_render_levels(_handles(levels), len(levels), views, n_views, ctypes.byref(outputs),
                                  ctypes.byref(opts) if opts is not None else None, stream), "lfp_render_levels")


def lfp_render_backward_levels(levels, views, n_views, grad_rgb, cls, aux_probe, aux_uv, grad_radiance, reduction,
                               stream) -> None:
    """grad_radiance: one device pointer (or None) per level."""
    gp = (ctypes.c_void_p * len(levels))(*grad_radiance)
    _check(_lib.lfp_render_backward_levels(_handles(levels), len(levels), views, n_views, grad_rgb, cls, aux_probe,
                                           aux_uv, gp, reduction, stream), "lfp_render_backward_levels")


def lfp_set_radiance(grid, dev_radiance, stream) -> None:
    _check(_lib.lfp_set_radiance(grid, dev_radiance, stream), "lfp_set_radiance")


def lfp_check_flags(grid, stream) -> int:
    return _check(_lib.lfp_check_flags(grid, stream), "lfp_check_flags")


def lfp_grid_bytes(desc: lfp_grid_desc) -> int:
    b = ctypes.c_ulonglong()
    _check(_lib.lfp_grid_bytes(ctypes.byref(desc), ctypes.byref(b)), "lfp_grid_bytes")
    return b.value


def lfp_skip_blocks(desc: lfp_grid_desc) -> list:
    """The block sides of the grid's skip levels, ascending."""
    ks = (ctypes.c_int * LFP_MAX_SKIP_LEVELS)()
    n = ctypes.c_int()
    _check(_lib.lfp_skip_blocks(ctypes.byref(desc), ks, ctypes.byref(n)), "lfp_skip_blocks")
    return list(ks[:n.value])


def raw_call(name: str, *args) -> int:
    """Call an entry point and return its raw status (for argument-validation tests)."""
    return getattr(_lib, name)(*args)
