"""FP64 CPU oracle for the light-field-probe ray tracer -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline /
reference arm may import this package. The product path (the C-ABI library
and its Python binding) never imports it and shares no code with it.

The arithmetic lives in ``lfp_oracle.c`` (double precision, one pixel at a
time, OpenMP over pixels); this module only marshals numpy arrays. Every
function cites the passage of Liu, Nowrouzezahrai & McGuire, "Real-Time Scene
Reconstruction using Light Field Probes" (arXiv 2507.14624) that it follows;
the C file's header lists the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfp_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")

MISS, HIT, UNKNOWN = 0, 1, 2
MARCH_FLAT, MARCH_HIER, MARCH_HIER_SHORTCUT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction: same results on x86-64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
                        "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"], check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("origin", ctypes.c_double * 3), ("spacing", ctypes.c_double),
                ("N", ctypes.c_int), ("M", ctypes.c_int),
                ("thickness_rel", ctypes.c_double), ("eye_eps", ctypes.c_double),
                ("march_mode", ctypes.c_int), ("eye_nearest", ctypes.c_int), ("traversal", ctypes.c_int)]


class _Probes(ctypes.Structure):
    _fields_ = [("dist", ctypes.c_void_p), ("normal", ctypes.c_void_p), ("radiance", ctypes.c_void_p),
                ("mip_min", ctypes.c_void_p), ("mip_max", ctypes.c_void_p)]


class _View(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_double * 3), ("right", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("fwd", ctypes.c_double * 3), ("fov_y", ctypes.c_double), ("W", ctypes.c_int),
                ("H", ctypes.c_int)]


class _Cell(ctypes.Structure):
    _fields_ = [("c", ctypes.c_int * 3), ("t_in", ctypes.c_double), ("t_out", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, ll, i, d = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_double
        G, Pr, V = ctypes.POINTER(_Grid), ctypes.POINTER(_Probes), ctypes.POINTER(_View)
        sig = {
            "orc_oct_encode_n": ([ll, vp, vp], None),
            "orc_oct_decode_n": ([ll, vp, vp], None),
            "orc_mirror_texel": ([i, vp, vp], None),
            "orc_build_mip": ([i, i, i, vp, vp, vp], None),
            "orc_split_segments": ([vp, vp, vp, d, d, vp], i),
            "orc_grid_cells": ([G, vp, vp, vp, i], i),
            "orc_cage_order": ([G, vp, vp, vp], None),
            "orc_render": ([G, Pr, V, ll, vp, vp, vp, vp, vp, vp, vp, vp], None),
            "orc_trace_rays": ([G, Pr, ll, vp, vp, vp, vp, vp, vp, vp, vp], None),
            "orc_trace_one_probe": ([G, Pr, i, vp, vp, d, d, vp, vp, vp], i),
            "orc_walk_segment": ([vp, vp, d, d, i, i, vp, vp], i),
            "orc_backward": ([G, ll, vp, vp, vp, vp, vp], None),
            "orc_bilinear_taps": ([i, vp, vp, vp, vp], None),
            "orc_num_threads": ([], i),
            "orc_splat_probes": ([ll, vp, vp, vp, i, vp, i, ctypes.c_float, vp, vp, vp, vp, vp, vp], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


# ---------------------------------------------------------------------------
# octahedral map (Sec. 3)
# ---------------------------------------------------------------------------

def oct_encode(d: np.ndarray) -> np.ndarray:
    """Direction(s) [..., 3] -> octahedral square point(s) [..., 2] in [-1, 1]^2."""
    d = _f64(d)
    shp = d.shape[:-1]
    d = d.reshape(-1, 3)
    out = np.empty((len(d), 2), np.float64)
    _load().orc_oct_encode_n(len(d), _p(d), _p(out))
    return out.reshape(*shp, 2)


def oct_decode(p: np.ndarray) -> np.ndarray:
    """Octahedral square point(s) [..., 2] -> unit direction(s) [..., 3]."""
    p = _f64(p)
    shp = p.shape[:-1]
    p = p.reshape(-1, 2)
    out = np.empty((len(p), 3), np.float64)
    _load().orc_oct_decode_n(len(p), _p(p), _p(out))
    return out.reshape(*shp, 3)


def num_threads() -> int:
    """Host threads the oracle's OpenMP loops use."""
    return int(_load().orc_num_threads())


def mirror_texel(R: int, i: int, j: int):
    ci, cj = ctypes.c_int(i), ctypes.c_int(j)
    _load().orc_mirror_texel(R, ctypes.byref(ci), ctypes.byref(cj))
    return ci.value, cj.value


def bilinear_taps(N: int, uv):
    uv = _f64(uv)
    ti = np.empty(4, np.int32)
    tj = np.empty(4, np.int32)
    w = np.empty(4, np.float64)
    _load().orc_bilinear_taps(N, _p(uv), _p(ti), _p(tj), _p(w))
    return ti, tj, w


def build_mip(dist: np.ndarray, M: int):
    """Per-block min and max of the distance maps (low-resolution map, Sec. 5.1)."""
    dist = np.ascontiguousarray(dist, np.float32)
    P, N, _ = dist.shape
    mn = np.empty((P, M, M), np.float32)
    mx = np.empty((P, M, M), np.float32)
    _load().orc_build_mip(P, N, M, _p(dist), _p(mn), _p(mx))
    return mn, mx


def split_segments(X, w, O, t0, t1):
    b = np.empty(5, np.float64)
    n = _load().orc_split_segments(_p(_f64(X)), _p(_f64(w)), _p(_f64(O)), t0, t1, _p(b))
    return [(b[k], b[k + 1]) for k in range(n)]


def walk_segment(Y0, w, ta, tb, R, max_texels=100000):
    """Texels (i, j) and their t-intervals along one octant segment at resolution R."""
    ij = np.empty((max_texels, 2), np.int32)
    tt = np.empty((max_texels, 2), np.float64)
    n = _load().orc_walk_segment(_p(_f64(Y0)), _p(_f64(w)), ta, tb, R, max_texels, _p(ij), _p(tt))
    return ij[:n].copy(), tt[:n].copy()


# ---------------------------------------------------------------------------
# the tracer
# ---------------------------------------------------------------------------

class Oracle:
    """FP64 tracer over one probe grid.

    grid: an object with nx, ny, nz, origin, spacing, N, M (e.g. synth.Grid).
    dist [P][N][N], normal [P][N][N][3], radiance [P][N][N][3]: float32 maps.
    """

    def __init__(self, grid, dist, normal, radiance, thickness_rel=1.0, eye_eps=None,
                 march=MARCH_HIER, eye_nearest=False, traversal=0):
        self.grid = grid
        self.dist = np.ascontiguousarray(dist, np.float32)
        self.normal = np.ascontiguousarray(normal, np.float32)
        self.radiance = np.ascontiguousarray(radiance, np.float32)
        self.mip_min, self.mip_max = build_mip(self.dist, grid.M)
        self.thickness_rel = float(thickness_rel)
        self.eye_eps = float(1e-6 * grid.spacing if eye_eps is None else eye_eps)
        self.march = march
        self.eye_nearest = int(bool(eye_nearest))
        self.traversal = int(traversal)

    def _g(self, march=None):
        g = _Grid()
        g.nx, g.ny, g.nz = self.grid.nx, self.grid.ny, self.grid.nz
        for a in range(3):
            g.origin[a] = float(self.grid.origin[a])
        g.spacing = float(self.grid.spacing)
        g.N, g.M = self.grid.N, self.grid.M
        g.thickness_rel = self.thickness_rel
        g.eye_eps = self.eye_eps
        g.march_mode = self.march if march is None else march
        g.eye_nearest = self.eye_nearest
        g.traversal = self.traversal
        return g

    def _pr(self):
        pr = _Probes()
        pr.dist, pr.normal, pr.radiance = (self.dist.ctypes.data, self.normal.ctypes.data,
                                           self.radiance.ctypes.data)
        pr.mip_min, pr.mip_max = self.mip_min.ctypes.data, self.mip_max.ctypes.data
        return pr

    @staticmethod
    def _v(view):
        v = _View()
        for a in range(3):
            v.pos[a], v.right[a], v.up[a], v.fwd[a] = view.pos[a], view.right[a], view.up[a], view.fwd[a]
        v.fov_y, v.W, v.H = view.fov_y, view.W, view.H
        return v

    def render(self, view, pixels=None, march=None, counters=False):
        """Trace the listed pixels (flat indices y*W + x; all when None) of one view.

        Returns a dict: rgb [n,3] f64, cls [n] u8, probe [n] i32, uv [n,2] f64,
        texel [n,2] i32 (fine texel that decided the HIT), t_hit [n] f64 and,
        when asked, counters [n,5] (coarse, fine, normal fetches, cells, probes).
        """
        if pixels is None:
            n = view.W * view.H
            pix = None
        else:
            pix = np.ascontiguousarray(pixels, np.int64)
            n = len(pix)
        out = {"rgb": np.zeros((n, 3)), "cls": np.zeros(n, np.uint8), "probe": np.zeros(n, np.int32),
               "uv": np.zeros((n, 2)), "texel": np.zeros((n, 2), np.int32), "t_hit": np.zeros(n)}
        cnt = np.zeros((n, 5), np.int64) if counters else None
        g, pr, v = self._g(march), self._pr(), self._v(view)
        _load().orc_render(ctypes.byref(g), ctypes.byref(pr), ctypes.byref(v), n, _p(pix),
                           _p(out["rgb"]), _p(out["cls"]), _p(out["probe"]), _p(out["uv"]),
                           _p(out["texel"]), _p(out["t_hit"]), _p(cnt))
        if counters:
            out["counters"] = cnt
        return out

    def trace_rays(self, X, W, march=None):
        """Trace arbitrary rays: origins X [n,3], directions W [n,3]."""
        X = _f64(X).reshape(-1, 3)
        W = _f64(W).reshape(-1, 3)
        n = len(X)
        out = {"rgb": np.zeros((n, 3)), "cls": np.zeros(n, np.uint8), "probe": np.zeros(n, np.int32),
               "uv": np.zeros((n, 2)), "texel": np.zeros((n, 2), np.int32), "t_hit": np.zeros(n)}
        g, pr = self._g(march), self._pr()
        _load().orc_trace_rays(ctypes.byref(g), ctypes.byref(pr), n, _p(X), _p(W), _p(out["rgb"]),
                               _p(out["cls"]), _p(out["probe"]), _p(out["uv"]), _p(out["texel"]),
                               _p(out["t_hit"]))
        return out

    def trace_one_probe(self, probe, X, w, t0, t1, march=None):
        """traceOneProbe over [t0, t1] (Appendix A): (class, texel, uv, t_hit)."""
        g, pr = self._g(march), self._pr()
        tex = np.empty(2, np.int32)
        uv = np.empty(2, np.float64)
        th = ctypes.c_double()
        c = _load().orc_trace_one_probe(ctypes.byref(g), ctypes.byref(pr), probe, _p(_f64(X)), _p(_f64(w)),
                                        t0, t1, _p(tex), _p(uv), ctypes.byref(th))
        return c, tex, uv, th.value

    def grid_cells(self, X, w, max_cells=1024):
        """Grid iterator (Sec. 4.3): [(cell ijk, t_in, t_out)] in ray order."""
        cells = (_Cell * max_cells)()
        n = _load().orc_grid_cells(ctypes.byref(self._g()), _p(_f64(X)), _p(_f64(w)), cells, max_cells)
        return [(tuple(cells[k].c), cells[k].t_in, cells[k].t_out) for k in range(n)]

    def cage_order(self, c, P):
        order = np.empty(8, np.int32)
        _load().orc_cage_order(ctypes.byref(self._g()), _p(np.asarray(c, np.int32)), _p(_f64(P)), _p(order))
        return order

    def backward(self, grad_rgb, cls, probe, uv):
        """Adjoint of render w.r.t. radiance: [P][N][N][3] f64 (sum over pixels)."""
        P, N = self.dist.shape[0], self.grid.N
        grad = np.zeros((P, N, N, 3), np.float64)
        g = _f64(grad_rgb).reshape(-1, 3)
        c = np.ascontiguousarray(cls, np.uint8)
        pb = np.ascontiguousarray(probe, np.int32)
        uv = _f64(uv).reshape(-1, 2)
        _load().orc_backward(ctypes.byref(self._g()), len(c), _p(g), _p(c), _p(pb), _p(uv), _p(grad))
        return grad


# ---------------------------------------------------------------------------
# multi-scale hierarchy
# ---------------------------------------------------------------------------

def probe_box(grid):
    """Closed box spanned by a grid's probes: [origin, origin + spacing (n - 1)]
    per axis, the float32 positions every consumer sees."""
    o = np.asarray(grid.origin, np.float32)
    s = np.float32(grid.spacing)
    n = np.array([grid.nx - 1, grid.ny - 1, grid.nz - 1], np.float32)
    return o.astype(np.float64), (o + s * n).astype(np.float32).astype(np.float64)


def pick_level(levels, X):
    """Level that traces a ray starting at X in a multi-scale hierarchy of
    probe grids (the multi-scale representation named in the abstract, the
    hierarchical scene representation of the teaser figure): the finest
    level (smallest spacing, ties to the lower index) whose probe box contains
    X; if none does, the coarsest (largest spacing, ties to the lower index)."""
    X = np.asarray(X, np.float64)
    best = None
    for k, g in enumerate(levels):
        lo, hi = probe_box(g)
        if np.all(X >= lo) and np.all(X <= hi) and (best is None or g.spacing < levels[best].spacing):
            best = k
    if best is None:
        for k, g in enumerate(levels):
            if best is None or g.spacing > levels[best].spacing:
                best = k
    return best


class Hierarchy:
    """FP64 tracer over a multi-scale hierarchy: one Oracle per level; every
    ray of a view starts at the camera, so the view is traced in the level
    pick_level gives for the camera position."""

    def __init__(self, levels, maps, **kw):
        self.levels = list(levels)
        self.oracles = [Oracle(g, *m, **kw) for g, m in zip(levels, maps)]

    def level_of(self, view):
        return pick_level(self.levels, view.pos)

    def render(self, view, pixels=None, **kw):
        k = self.level_of(view)
        out = self.oracles[k].render(view, pixels, **kw)
        out["level"] = k
        return out

    def backward(self, views, grad_rgb, cls, probe, uv):
        """Per-level radiance gradients ([P_l][N_l][N_l][3] f64) of the views'
        concatenated pixels (flat, in view order)."""
        grads = [np.zeros((o.dist.shape[0], g.N, g.N, 3)) for o, g in zip(self.oracles, self.levels)]
        off = 0
        for v in views:
            n = v.W * v.H
            k = self.level_of(v)
            sl = slice(off, off + n)
            grads[k] += self.oracles[k].backward(np.asarray(grad_rgb)[sl], np.asarray(cls)[sl],
                                                 np.asarray(probe)[sl], np.asarray(uv)[sl])
            off += n
        return grads


# ---------------------------------------------------------------------------
# probe maps from a point cloud
# ---------------------------------------------------------------------------

def splat_probes(xyz, rgb, probe_pos, N, normal=None, empty_dist=0.0, details=False):
    """Probe maps from a point cloud (Sec. 4.1 simulated probes, Sec. 5.1
    probe data generation), in double precision: per probe and texel the
    point nearest to the probe (ties to the lower point index); see
    lfp_oracle.c. xyz, rgb, normal: [n][3]; probe_pos [P][3]. Returns float32
    dist [P][N][N], normal [P][N][N][3] (the points' normals, or the incoming
    direction -v/|v| when normal is None), radiance [P][N][N][3]; with
    details=True also a dict: winner [P][N][N] int64 (-1 empty), decided
    [P][N][N] bool (float32 rounding of the builder's recipe cannot change
    the winner), dcand [P][N][N] float32 (least distance of a point that
    float32 rounding can put into the texel, inf if none)."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
    rgb = np.ascontiguousarray(rgb, np.float32).reshape(-1, 3)
    nrm = None if normal is None else np.ascontiguousarray(normal, np.float32).reshape(-1, 3)
    pos = np.ascontiguousarray(probe_pos, np.float32).reshape(-1, 3)
    P = len(pos)
    dist = np.empty((P, N, N), np.float32)
    nout = np.empty((P, N, N, 3), np.float32)
    rad = np.empty((P, N, N, 3), np.float32)
    win = dec = dc = None
    if details:
        win = np.empty((P, N, N), np.int64)
        dec = np.empty((P, N, N), np.uint8)
        dc = np.empty((P, N, N), np.float32)
    lib.orc_splat_probes(ctypes.c_longlong(len(xyz)), _p(xyz), _p(rgb), _p(nrm), P, _p(pos), N,
                         ctypes.c_float(empty_dist), _p(dist), _p(nout), _p(rad), _p(win), _p(dec), _p(dc))
    if details:
        return dist, nout, rad, {"winner": win, "decided": dec.astype(bool), "dcand": dc}
    return dist, nout, rad
