"""Seeded synthetic inputs for the light-field-probe tracer.

This module is the one input generator that both the FP64 oracle and the CUDA
path consume. It builds

* a scene of spheres and axis-aligned boxes inside a closed room, lit by
  directional lights (Lambertian, hard shadows cast by the objects);
* the probe grid and its octahedral probe maps (distance, surface normal,
  radiance), made by casting one ray per texel centre -- the stand-in for the
  paper's point-cloud projection (Sec. 5.1, Probe Data Generation);
* pinhole cameras (the ray (X, omega_1) of Sec. 3).

It holds no step of the probe tracer (no marching, classification or
radiance lookup). Random numbers come from SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_libsynth.so")
_SRC = os.path.join(_HERE, "raycast.c")

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 as published (golden-gamma increment, two xor-shift-multiply rounds)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


# ----------------------------------------------------------------------------
# build / load the C ray caster
# ----------------------------------------------------------------------------

def build(force: bool = False) -> str:
    """Compile raycast.c into _libsynth.so (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
               "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _SceneC(ctypes.Structure):
    _fields_ = [
        ("n_spheres", ctypes.c_int), ("spheres", ctypes.c_void_p),
        ("n_boxes", ctypes.c_int), ("boxes", ctypes.c_void_p),
        ("room", ctypes.c_void_p), ("wall_albedo", ctypes.c_void_p),
        ("n_lights", ctypes.c_int), ("lights", ctypes.c_void_p),
        ("ambient", ctypes.c_double),
        ("acc_dims", ctypes.c_int * 3), ("acc_lo", ctypes.c_void_p), ("acc_cell", ctypes.c_void_p),
        ("acc_start", ctypes.c_void_p), ("acc_items", ctypes.c_void_p),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        vp, ll, i = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int
        lib.syn_cast.argtypes = [ctypes.POINTER(_SceneC), ll, vp, vp, vp, vp, vp, vp]
        lib.syn_cast.restype = None
        lib.syn_probe_maps.argtypes = [ctypes.POINTER(_SceneC), i, vp, i, vp, vp, vp]
        lib.syn_probe_maps.restype = None
        lib.syn_texel_directions.argtypes = [i, vp]
        lib.syn_texel_directions.restype = None
        lib.syn_scan.argtypes = [ctypes.POINTER(_SceneC), vp, i, i, ctypes.c_double, ctypes.c_double, vp, vp, vp]
        lib.syn_scan.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------
# grid, scene, cameras
# ----------------------------------------------------------------------------

@dataclass
class Grid:
    """Probes at the vertices of a uniform 3D grid (Sec. 3, multiple probes)."""
    nx: int
    ny: int
    nz: int
    spacing: float
    N: int                     # full-resolution octahedral map side
    M: int                     # min/max mip side (N % M == 0)
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def n_probes(self) -> int:
        return self.nx * self.ny * self.nz

    def probe_positions(self) -> np.ndarray:
        """[P][3] float64, probe index = ix + nx*(iy + ny*iz). Positions are
        the float32 values origin + spacing*i, as every consumer sees them."""
        o = np.asarray(self.origin, dtype=np.float32)
        s = np.float32(self.spacing)
        pos = np.empty((self.n_probes, 3), dtype=np.float32)
        k = 0
        for iz in range(self.nz):
            for iy in range(self.ny):
                for ix in range(self.nx):
                    pos[k] = (o[0] + s * np.float32(ix), o[1] + s * np.float32(iy), o[2] + s * np.float32(iz))
                    k += 1
        return pos.astype(np.float64)

    def lo(self) -> np.ndarray:
        return np.asarray(self.origin, dtype=np.float64)

    def hi(self) -> np.ndarray:
        return self.lo() + self.spacing * np.array([self.nx - 1, self.ny - 1, self.nz - 1], dtype=np.float64)


@dataclass
class Scene:
    grid: Grid
    spheres: np.ndarray        # [ns][7]
    boxes: np.ndarray          # [nb][9]
    room: np.ndarray           # [6]
    wall_albedo: np.ndarray    # [6][3]
    lights: np.ndarray         # [nl][4]
    ambient: float
    seed: int
    accel: dict = field(default_factory=dict)

    def _cstruct(self) -> _SceneC:
        c = _SceneC()
        c.n_spheres = len(self.spheres)
        c.spheres = self.spheres.ctypes.data if len(self.spheres) else None
        c.n_boxes = len(self.boxes)
        c.boxes = self.boxes.ctypes.data if len(self.boxes) else None
        c.room = self.room.ctypes.data
        c.wall_albedo = self.wall_albedo.ctypes.data
        c.n_lights = len(self.lights)
        c.lights = self.lights.ctypes.data if len(self.lights) else None
        c.ambient = self.ambient
        if self.accel:
            a = self.accel
            for k in range(3):
                c.acc_dims[k] = int(a["dims"][k])
            c.acc_lo = a["lo"].ctypes.data
            c.acc_cell = a["cell"].ctypes.data
            c.acc_start = a["start"].ctypes.data
            c.acc_items = a["items"].ctypes.data
        self._keep = c  # keep struct alive with the arrays
        return c

    # ------------------------------------------------------------------
    def cast(self, origins: np.ndarray, dirs: np.ndarray):
        """Analytic nearest hit: returns (t, normal, radiance, prim_id)."""
        lib = _load()
        o = np.ascontiguousarray(origins, dtype=np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        n = len(o)
        t = np.empty(n, np.float64)
        nn = np.empty((n, 3), np.float64)
        rgb = np.empty((n, 3), np.float64)
        prim = np.empty(n, np.int32)
        lib.syn_cast(ctypes.byref(self._cstruct()), n, _ptr(o), _ptr(d), _ptr(t), _ptr(nn), _ptr(rgb), _ptr(prim))
        return t, nn, rgb, prim

    def probe_maps(self, probe_pos: np.ndarray | None = None, N: int | None = None, normal_mode: str = "surface"):
        """Probe maps for every probe of the grid (or the given positions):
        dist [P][N][N] f32, normal [P][N][N][3] f32, radiance [P][N][N][3] f32.

        normal_mode "surface": the geometric normal at the texel's surface
        point; "incoming": the direction in which light from that point
        arrives at the probe (point -> probe, minus the texel's direction),
        the content Sec. 5.1 gives its normal map."""
        if normal_mode not in ("surface", "incoming"):
            raise ValueError(normal_mode)
        lib = _load()
        pos = self.grid.probe_positions() if probe_pos is None else np.asarray(probe_pos, np.float64)
        pos = np.ascontiguousarray(pos.reshape(-1, 3))
        N = self.grid.N if N is None else N
        P = len(pos)
        dist = np.empty((P, N, N), np.float32)
        nrm = np.empty((P, N, N, 3), np.float32)
        rad = np.empty((P, N, N, 3), np.float32)
        lib.syn_probe_maps(ctypes.byref(self._cstruct()), P, _ptr(pos), N, _ptr(dist), _ptr(nrm), _ptr(rad))
        if normal_mode == "incoming":
            nrm[:] = -texel_directions(N).astype(np.float32)[None]
        return dist, nrm, rad

    def distance_to_objects(self, p: np.ndarray) -> float:
        """Signed-ish clearance: min over objects of distance from p (0 inside a box)."""
        best = math.inf
        for s in self.spheres:
            best = min(best, float(np.linalg.norm(p - s[:3]) - s[3]))
        for b in self.boxes:
            q = np.maximum(np.maximum(b[:3] - p, p - b[3:6]), 0.0)
            best = min(best, float(np.linalg.norm(q)) if np.any(q > 0) else -1.0)
        return best


def texel_directions(N: int) -> np.ndarray:
    """[N][N][3] unit texel-centre directions of the probe-map format."""
    out = np.empty((N, N, 3), np.float64)
    _load().syn_texel_directions(N, _ptr(out))
    return out


def _box_clearance(b, p):
    q = np.maximum(np.maximum(b[:3] - p, p - b[3:6]), 0.0)
    return float(np.linalg.norm(q)) if np.any(q > 0) else -1.0


def _build_accel(spheres: np.ndarray, boxes: np.ndarray, room: np.ndarray, cell: float) -> dict:
    lo = room[:3].astype(np.float64)
    ext = room[3:] - room[:3]
    dims = np.maximum(1, np.ceil(ext / cell).astype(np.int64))
    cs = ext / dims
    buckets = [[] for _ in range(int(np.prod(dims)))]

    def add(obj_id, bmin, bmax):
        c0 = np.clip(np.floor((bmin - lo) / cs).astype(int), 0, dims - 1)
        c1 = np.clip(np.floor((bmax - lo) / cs).astype(int), 0, dims - 1)
        for z in range(c0[2], c1[2] + 1):
            for y in range(c0[1], c1[1] + 1):
                for x in range(c0[0], c1[0] + 1):
                    buckets[x + dims[0] * (y + dims[1] * z)].append(obj_id)

    for k, s in enumerate(spheres):
        add(k, s[:3] - s[3] - 1e-9, s[:3] + s[3] + 1e-9)
    for k, b in enumerate(boxes):
        add(len(spheres) + k, b[:3] - 1e-9, b[3:6] + 1e-9)
    start = np.zeros(len(buckets) + 1, np.int32)
    for k, bkt in enumerate(buckets):
        start[k + 1] = start[k] + len(bkt)
    items = np.array([i for bkt in buckets for i in bkt] or [0], np.int32)
    return {"dims": dims.astype(np.int32), "lo": np.ascontiguousarray(lo), "cell": np.ascontiguousarray(cs),
            "start": start, "items": items}


def make_scene(grid: Grid, n_spheres: int, n_boxes: int, light_intensities, seed: int,
               ambient: float = 0.1, room_margin: float | None = None, clearance: float = 0.02,
               accel_cell: float | None = None, size_scale: float = 1.0) -> Scene:
    """Random scene around a probe grid.

    * Room: the grid's bounding box grown by half a spacing on each side,
      inward-facing walls with albedo U[0,1]^3.
    * Spheres: radius U[0.05, 0.2], centre uniform in the room.
    * Boxes: axis-aligned, half-extents U[0.05, 0.25] * (spacing / 0.5), each
      capped at 0.4 * spacing, centre uniform in the room.
    * Objects are redrawn while one contains a probe or comes within
      `clearance` of one. Albedo U[0,1]^3.
    * Lights: directions uniform on the upper hemisphere.
    * size_scale multiplies every radius and half-extent (denser scenes of
      smaller objects).
    """
    rng = SplitMix64(seed)
    margin = 0.5 * grid.spacing if room_margin is None else room_margin
    room = np.concatenate([grid.lo() - margin, grid.hi() + margin]).astype(np.float64)
    probes = grid.probe_positions()
    wall_albedo = np.array([[rng.uniform() for _ in range(3)] for _ in range(6)], np.float64)

    def far_from_probes_sphere(c, r):
        d = np.linalg.norm(probes - c, axis=1) - r
        return bool(np.all(d >= clearance))

    def far_from_probes_box(b):
        q = np.maximum(np.maximum(b[:3] - probes, probes - b[3:6]), 0.0)
        d = np.linalg.norm(q, axis=1)
        inside = np.all((probes >= b[:3]) & (probes <= b[3:6]), axis=1)
        return bool(np.all(d >= clearance) and not np.any(inside))

    spheres = []
    while len(spheres) < n_spheres:
        r = rng.uniform(0.05, 0.2) * size_scale
        c = np.array([rng.uniform(room[a], room[a + 3]) for a in range(3)])
        alb = [rng.uniform() for _ in range(3)]
        if far_from_probes_sphere(c, r):
            spheres.append([*c, r, *alb])
    boxes = []
    scale = grid.spacing / 0.5
    cap = 0.4 * grid.spacing
    while len(boxes) < n_boxes:
        h = np.array([min(rng.uniform(0.05, 0.25) * scale, cap) * size_scale for _ in range(3)])
        c = np.array([rng.uniform(room[a], room[a + 3]) for a in range(3)])
        alb = [rng.uniform() for _ in range(3)]
        b = np.array([*(c - h), *(c + h)])
        if far_from_probes_box(b):
            boxes.append([*b, *alb])
    lights = []
    for inten in light_intensities:
        z = rng.uniform()
        phi = rng.uniform(0.0, 2.0 * math.pi)
        s = math.sqrt(max(0.0, 1.0 - z * z))
        lights.append([s * math.cos(phi), s * math.sin(phi), z, float(inten)])
    sph = np.ascontiguousarray(np.array(spheres, np.float64).reshape(-1, 7))
    bxs = np.ascontiguousarray(np.array(boxes, np.float64).reshape(-1, 9))
    accel = {}
    if accel_cell is not None and (len(sph) + len(bxs)) > 0:
        accel = _build_accel(sph, bxs, room, accel_cell)
    return Scene(grid=grid, spheres=sph, boxes=bxs, room=room, wall_albedo=wall_albedo,
                 lights=np.ascontiguousarray(np.array(lights, np.float64).reshape(-1, 4)),
                 ambient=ambient, seed=seed, accel=accel)


@dataclass
class View:
    """Pinhole camera: ray through pixel (x, y) leaves `pos` along
    fwd + a*right + b*up, a = ((x+.5)/W*2-1)*tan(fov_y/2)*W/H,
    b = (1-(y+.5)/H*2)*tan(fov_y/2); fov_y is the vertical field of view."""
    pos: tuple
    right: tuple
    up: tuple
    fwd: tuple
    fov_y: float
    W: int
    H: int

    @property
    def n_pixels(self) -> int:
        return self.W * self.H


def look_view(pos, yaw: float, pitch: float, fov_y_deg: float, W: int, H: int) -> View:
    cp, sp = math.cos(pitch), math.sin(pitch)
    fwd = np.array([cp * math.cos(yaw), cp * math.sin(yaw), sp])
    right = np.array([math.sin(yaw), -math.cos(yaw), 0.0])
    up = np.cross(right, fwd)
    f32 = lambda v: tuple(float(np.float32(x)) for x in v)  # noqa: E731 - every consumer sees float32
    return View(pos=f32(pos), right=f32(right), up=f32(up), fwd=f32(fwd),
                fov_y=float(np.float32(math.radians(fov_y_deg))), W=W, H=H)


def random_view(scene: Scene, seed: int, W: int, H: int, fov_y_deg: float, clearance: float = 0.02) -> View:
    """Camera uniform in the probe cage shrunk by 10% about its centre, redrawn
    while within `clearance` of an object; yaw U[0, 2pi), pitch U[-30, 30] deg."""
    rng = SplitMix64(seed)
    lo, hi = scene.grid.lo(), scene.grid.hi()
    c, h = 0.5 * (lo + hi), 0.5 * (hi - lo) * 0.9
    while True:
        p = np.array([rng.uniform(c[a] - h[a], c[a] + h[a]) for a in range(3)])
        yaw = rng.uniform(0.0, 2.0 * math.pi)
        pitch = math.radians(rng.uniform(-30.0, 30.0))
        pf = np.array([float(np.float32(x)) for x in p])
        if scene.distance_to_objects(pf) >= clearance:
            return look_view(pf, yaw, pitch, fov_y_deg, W, H)


def catmull_rom_views(scene: Scene, seed: int, sizes, fov_y_deg: float, n_ctrl: int = 8,
                      clearance: float = 0.02) -> list:
    """len(sizes) cameras along a seeded Catmull-Rom path through the cage.
    Control points are uniform in the shrunk cage (clear of objects); each
    camera looks along the path tangent (pitch clamped to +-30 deg) plus a
    seeded yaw jitter; samples that fall within `clearance` of an object are
    moved along the path until clear."""
    rng = SplitMix64(seed)
    lo, hi = scene.grid.lo(), scene.grid.hi()
    c, h = 0.5 * (lo + hi), 0.5 * (hi - lo) * 0.9
    ctrl = []
    while len(ctrl) < n_ctrl:
        p = np.array([rng.uniform(c[a] - h[a], c[a] + h[a]) for a in range(3)])
        if scene.distance_to_objects(p) >= 0.05:
            ctrl.append(p)
    ctrl = np.array(ctrl)

    def curve(s):
        seg = min(int(s), n_ctrl - 4)
        u = s - seg
        p0, p1, p2, p3 = ctrl[seg:seg + 4]
        pos = 0.5 * ((2 * p1) + (-p0 + p2) * u + (2 * p0 - 5 * p1 + 4 * p2 - p3) * u * u
                     + (-p0 + 3 * p1 - 3 * p2 + p3) * u ** 3)
        tan = 0.5 * ((-p0 + p2) + 2 * (2 * p0 - 5 * p1 + 4 * p2 - p3) * u
                     + 3 * (-p0 + 3 * p1 - 3 * p2 + p3) * u * u)
        return np.clip(pos, c - h, c + h), tan

    views = []
    n = len(sizes)
    span = n_ctrl - 3
    for k, (W, H) in enumerate(sizes):
        s = span * (k + 0.5) / n
        for _ in range(1000):
            pos, tan = curve(min(s, span - 1e-9))
            pf = np.array([float(np.float32(x)) for x in pos])
            if scene.distance_to_objects(pf) >= clearance:
                break
            s = (s + 0.01) % span
        t = tan / (np.linalg.norm(tan) + 1e-12)
        yaw = math.atan2(t[1], t[0]) + rng.uniform(-0.5, 0.5)
        pitch = max(-math.radians(30.0), min(math.radians(30.0), math.asin(max(-1.0, min(1.0, t[2])))))
        views.append(look_view(pf, yaw, pitch, fov_y_deg, W, H))
    return views


# ----------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------

BATCH_SIZES = [(640, 480), (1280, 720), (1920, 1080), (3840, 2160)]


def workload(name: str):
    """Return (scene, views, info) for a named synthetic workload.

    tiny     2x2x2 probes, spacing 1.0, N=64, M=16; 8 spheres + 2 boxes, one
             light (1.0); one 128x128 view, 60 deg vertical FOV; seed 1.
    room     4x4x4 probes, spacing 0.5, N=256, M=16; 64 spheres + 16 boxes,
             two lights (0.7, 0.3); one 1920x1080 view, 70 deg; seed 2.
    batched  8x8x4 probes, spacing 0.5, N=512, M=32; 256 spheres + 64 boxes,
             two lights; 32 views with sizes drawn from 640x480 .. 3840x2160
             along a Catmull-Rom path (seed 303); scene seed 3.
    fit      the room grid with seed 4 and 64 views of 800x800 (70 deg).
    few      2x2x1 probes (the 4-probe scenario of Sec. 4.3), spacing 1.0,
             N=256, M=16; 16 spheres + 4 boxes, two lights; one 1920x1080
             view, 70 deg; seed 6.
    """
    if name == "tiny":
        g = Grid(2, 2, 2, 1.0, 64, 16)
        sc = make_scene(g, 8, 2, [1.0], seed=1)
        views = [random_view(sc, 101, 128, 128, 60.0)]
    elif name == "room":
        g = Grid(4, 4, 4, 0.5, 256, 16)
        sc = make_scene(g, 64, 16, [0.7, 0.3], seed=2, accel_cell=0.25)
        views = [random_view(sc, 102, 1920, 1080, 70.0)]
    elif name == "batched":
        g = Grid(8, 8, 4, 0.5, 512, 32)
        sc = make_scene(g, 256, 64, [0.7, 0.3], seed=3, accel_cell=0.25)
        rng = SplitMix64(303)
        sizes = [BATCH_SIZES[int(rng.uniform() * 4) % 4] for _ in range(32)]
        views = catmull_rom_views(sc, 303, sizes, 70.0)
    elif name == "fit":
        g = Grid(4, 4, 4, 0.5, 256, 16)
        sc = make_scene(g, 64, 16, [0.7, 0.3], seed=4, accel_cell=0.25)
        views = [random_view(sc, 104 + 1000 * k, 800, 800, 70.0) for k in range(64)]
    elif name == "few":
        g = Grid(2, 2, 1, 1.0, 256, 16)
        sc = make_scene(g, 16, 4, [0.7, 0.3], seed=6)
        views = [random_view(sc, 106, 1920, 1080, 70.0)]
    else:
        raise ValueError(f"unknown workload {name!r}")
    return sc, views


# ---------------------------------------------------------------------------
# multi-scale hierarchy: nested probe grids over a street-grid scene
# ---------------------------------------------------------------------------

def multiscale_levels(scale: int = 1):
    """Three nested probe grids, coarse to fine (N and M divided by `scale`):

    L0 16x16x4 at spacing 2.0,   N=128, M=8,  origin (0, 0, 0):        x, y in [0, 30]
    L1 16x16x4 at spacing 0.5,   N=256, M=16, origin (11, 11, 0.5):    x, y in [11, 18.5]
    L2  8x8x4  at spacing 0.125, N=512, M=32, origin (14.5, 14.5, 0.5): x, y in [14.5, 15.375]
    """
    def g(nx, ny, nz, sp, N, M, o):
        N, M = N // scale, max(2, M // scale)
        return Grid(nx, ny, nz, sp, N, M, o)
    return [g(16, 16, 4, 2.0, 128, 8, (0.0, 0.0, 0.0)),
            g(16, 16, 4, 0.5, 256, 16, (11.0, 11.0, 0.5)),
            g(8, 8, 4, 0.125, 512, 32, (14.5, 14.5, 0.5))]


def street_scene(levels, n_spheres: int = 1024, seed: int = 5, lights=(0.7, 0.3), ambient: float = 0.1,
                 clearance: float = 0.02) -> Scene:
    """Street-grid scene around nested probe grids (levels[0] the outermost).

    * Room: levels[0]'s box grown by half its spacing; the floor is its lower z.
    * 64 x 64 lots at pitch 0.5 over the room's floor, centres at odd multiples
      of 0.25, one box per lot standing on the floor: footprint half-extents
      U[0.08, 0.22] (so no box reaches an x or y that is a multiple of 0.5,
      where the two outer levels' probes sit); lots in every 8th pair of rows
      and columns are streets (height U[0.1, 0.6]), the rest buildings
      (U[0.5, 6.0]); lots under the innermost level's box are a plaza (height
      U[0.05, 0.4], below its lowest probe).
    * Spheres radius U[0.05, 0.2], centre uniform in the room, redrawn while
      within `clearance` of any probe of any level. Albedo U[0,1]^3; lights
      directional, uniform on the upper hemisphere.
    """
    rng = SplitMix64(seed)
    g0 = levels[0]
    margin = 0.5 * g0.spacing
    room = np.concatenate([g0.lo() - margin, g0.hi() + margin]).astype(np.float64)
    wall_albedo = np.array([[rng.uniform() for _ in range(3)] for _ in range(6)], np.float64)
    probes = np.concatenate([g.probe_positions() for g in levels])
    inner_lo, inner_hi = levels[-1].lo(), levels[-1].hi()
    n_lots = int(round((room[3] - room[0]) / 0.5))
    boxes = []
    for j in range(n_lots):
        for i in range(n_lots):
            c = np.array([room[0] + 0.25 + 0.5 * i, room[1] + 0.25 + 0.5 * j])
            hx, hy = rng.uniform(0.08, 0.22), rng.uniform(0.08, 0.22)
            street = (i % 8) in (3, 4) or (j % 8) in (3, 4)
            plaza = (c[0] + 0.25 >= inner_lo[0] - 0.25 and c[0] - 0.25 <= inner_hi[0] + 0.25 and
                     c[1] + 0.25 >= inner_lo[1] - 0.25 and c[1] - 0.25 <= inner_hi[1] + 0.25)
            h = rng.uniform(0.05, 0.4) if plaza else (rng.uniform(0.1, 0.6) if street else rng.uniform(0.5, 6.0))
            alb = [rng.uniform() for _ in range(3)]
            boxes.append([c[0] - hx, c[1] - hy, room[2], c[0] + hx, c[1] + hy, room[2] + h, *alb])
    spheres = []
    while len(spheres) < n_spheres:
        r = rng.uniform(0.05, 0.2)
        c = np.array([rng.uniform(room[a], room[a + 3]) for a in range(3)])
        alb = [rng.uniform() for _ in range(3)]
        if np.all(np.linalg.norm(probes - c, axis=1) - r >= clearance):
            spheres.append([*c, r, *alb])
    lts = []
    for inten in lights:
        z = rng.uniform()
        phi = rng.uniform(0.0, 2.0 * math.pi)
        s = math.sqrt(max(0.0, 1.0 - z * z))
        lts.append([s * math.cos(phi), s * math.sin(phi), z, float(inten)])
    sph = np.ascontiguousarray(np.array(spheres, np.float64).reshape(-1, 7))
    bxs = np.ascontiguousarray(np.array(boxes, np.float64).reshape(-1, 9))
    return Scene(grid=g0, spheres=sph, boxes=bxs, room=room, wall_albedo=wall_albedo,
                 lights=np.ascontiguousarray(np.array(lts, np.float64).reshape(-1, 4)), ambient=ambient,
                 seed=seed, accel=_build_accel(sph, bxs, room, 0.5))


def level_scene(scene: Scene, grid: Grid) -> Scene:
    """The same scene with another probe grid (for its probe maps and cameras)."""
    from dataclasses import replace
    return replace(scene, grid=grid)


def _box_contains(g: Grid, p, shrink: float = 0.0) -> bool:
    lo, hi = g.lo(), g.hi()
    c, h = 0.5 * (lo + hi), 0.5 * (hi - lo) * (1.0 - shrink)
    return bool(np.all(p >= c - h) and np.all(p <= c + h))


def multiscale_views(scene: Scene, levels, seed: int, n_views: int, sizes, fov_y_deg: float = 70.0,
                     clearance: float = 0.05):
    """Views cycling over the levels: view k starts inside level k % L's probe
    box shrunk by 10 % and outside the next finer level's box, so every level
    is the finest one containing some cameras; yaw U[0, 2pi), pitch
    U[-30, 30] deg, redrawn while within `clearance` of an object."""
    rng = SplitMix64(seed)
    views = []
    for k in range(n_views):
        lev = k % len(levels)
        g = levels[lev]
        lo, hi = g.lo(), g.hi()
        c, h = 0.5 * (lo + hi), 0.5 * (hi - lo) * 0.9
        W, H = sizes[k % len(sizes)]
        while True:
            p = np.array([float(np.float32(rng.uniform(c[a] - h[a], c[a] + h[a]))) for a in range(3)])
            yaw = rng.uniform(0.0, 2.0 * math.pi)
            pitch = math.radians(rng.uniform(-30.0, 30.0))
            if lev + 1 < len(levels) and _box_contains(levels[lev + 1], p):
                continue
            if scene.distance_to_objects(p) >= clearance:
                views.append(look_view(p, yaw, pitch, fov_y_deg, W, H))
                break
    return views


def multiscale_workload(scale: int = 1, n_views: int = 64):
    """(scene, levels, views): the street-grid scene (4096 boxes, 1024
    spheres, seed 5), the three nested levels and `n_views` mixed-resolution
    views (sizes drawn from 640x480 .. 3840x2160 with seed 305, divided by
    `scale`; cameras seed 505)."""
    levels = multiscale_levels(scale)
    sc = street_scene(levels, seed=5)
    rng = SplitMix64(305)
    sizes = [BATCH_SIZES[int(rng.uniform() * 4) % 4] for _ in range(n_views)]
    sizes = [(max(1, W // scale), max(1, H // scale)) for W, H in sizes]
    views = multiscale_views(sc, levels, 505, n_views, sizes)
    return sc, levels, views


# ---------------------------------------------------------------------------
# point clouds: simulated laser scans (the stand-in for the FARO captures)
# ---------------------------------------------------------------------------

def scan(scene: Scene, positions, n_dirs: int, seed: int, vertical_deg: float = 300.0):
    """Point cloud of one laser scan per position (Sec. 5.2: the scanner
    turns 360 deg horizontally while its mirror sweeps `vertical_deg`
    vertically, so a cone of 360 - vertical_deg deg under it stays unseen).
    About n_dirs directions per scan on an (azimuth, polar angle) grid with
    equal angular steps and a seeded azimuth phase, recorded column by column
    as a scanner writes them; every ray's nearest hit is a point with its
    radiance and surface normal. Returns float32 arrays xyz [n][3], rgb
    [n][3], normal [n][3] (scans concatenated in order)."""
    lib = _load()
    rng = SplitMix64(seed)
    theta_max = math.radians(vertical_deg / 2.0)
    n_el = max(1, int(round(math.sqrt(n_dirs * theta_max / (2.0 * math.pi)))))
    n_az = max(1, n_dirs // n_el)
    out = {"xyz": [], "rgb": [], "normal": []}
    for p in np.asarray(positions, np.float64).reshape(-1, 3):
        n = n_az * n_el
        xyz = np.zeros((n, 3), np.float32)
        rgb = np.zeros((n, 3), np.float32)
        nrm = np.zeros((n, 3), np.float32)
        pos = np.ascontiguousarray(p)
        lib.syn_scan(ctypes.byref(scene._cstruct()), _ptr(pos), n_az, n_el, rng.uniform(0.0, 2.0 * math.pi),
                     theta_max, _ptr(xyz), _ptr(rgb), _ptr(nrm))
        out["xyz"].append(xyz)
        out["rgb"].append(rgb)
        out["normal"].append(nrm)
    return {k: np.ascontiguousarray(np.concatenate(v)) for k, v in out.items()}


def scan_positions(scene: Scene, n: int, seed: int, clearance: float = 0.05):
    """Scanner positions uniform in the probe cage, redrawn near objects."""
    rng = SplitMix64(seed)
    lo, hi = scene.grid.lo(), scene.grid.hi()
    out = []
    while len(out) < n:
        p = np.array([rng.uniform(lo[a], hi[a]) for a in range(3)])
        if scene.distance_to_objects(p) >= clearance:
            out.append(p)
    return np.array(out)
