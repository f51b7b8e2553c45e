"""Pins for the oracle's paper-faithful variants: the traversal Sec. 4.3 gives
for fewer than 8 probes, the eye-aligned texel fetch of Appendix A
traceOneProbe, and the normal-map content of Sec. 5.1 (incoming directions)."""
import numpy as np
import pytest

import oracle
import synth
from conftest import camera_rays
from test_oracle_trace import _within_one_texel

FEW_GRIDS = [(2, 1, 1), (2, 2, 1), (2, 2, 2)]


def _cam(sc, seed, W=64, H=48, fov=60.0):
    """A camera inside the room, off the probe planes (clear of objects)."""
    rng = np.random.default_rng(seed)
    lo, hi = sc.grid.lo() - 0.3 * sc.grid.spacing, sc.grid.hi() + 0.3 * sc.grid.spacing
    while True:
        p = np.float32(rng.uniform(lo, hi)).astype(np.float64)
        if sc.distance_to_objects(p) > 0.05:
            return synth.look_view(p, rng.uniform(0, 2 * np.pi), rng.uniform(-0.5, 0.5), fov, W, H)


@pytest.mark.parametrize("dims", FEW_GRIDS)
def test_nearest_mode_in_an_empty_room_hits_with_the_nearest_probe(dims):
    """Empty closed room: every probe sees every wall point, so the probe
    nearest to the eye (Sec. 4.3, 'start from the probe that is closest to
    the eye') decides the pixel unless it sees the wall nearly edge-on, where
    the stored distance changes by more than the crossing thickness from one
    texel to the next and the ray passes behind (UNKNOWN, next probe; measured
    92-100 % nearest on these cameras). Every pixel is a HIT whose texel is
    within one texel of oct(T - O), T the true hit."""
    g = synth.Grid(*dims, 1.0, 64, 16)
    sc = synth.make_scene(g, 0, 0, [1.0], seed=8)
    d, n, r = sc.probe_maps()
    for k in range(3):
        v = _cam(sc, 40 + k)
        res = oracle.Oracle(g, d, n, r, traversal=1).render(v)
        assert np.all(res["cls"] == oracle.HIT)
        P = g.probe_positions()
        nearest = int(np.argmin(np.linalg.norm(P - np.array(v.pos), axis=1)))
        assert np.mean(res["probe"] == nearest) >= 0.9
        X, D = camera_rays(v)
        t, _, _, _ = sc.cast(X, D)
        p = oracle.oct_encode(X + t[:, None] * D - P[res["probe"]])
        want = np.clip(np.floor((p + 1) / 2 * g.N).astype(int), 0, g.N - 1)
        assert np.all(_within_one_texel(g.N, res["texel"], want))


@pytest.mark.parametrize("dims", FEW_GRIDS)
def test_nearest_mode_falls_through_miss_and_unknown_in_distance_order(dims):
    """Brute force over the probes: each probe traced alone over the whole ray
    [0, inf); the result is the first HIT in order of distance to the eye
    (numpy argsort, ties to the lower index); with no HIT it is UNKNOWN if any
    probe said UNKNOWN, else MISS."""
    g = synth.Grid(*dims, 1.0, 32, 8)
    sc = synth.make_scene(g, 6, 2, [1.0], seed=9)
    d, n, r = sc.probe_maps()
    o = oracle.Oracle(g, d, n, r, traversal=1)
    P = g.probe_positions()
    n_fell_through = 0
    for k in range(3):
        v = _cam(sc, 60 + k, 24, 18)
        res = o.render(v)
        X, D = camera_rays(v)
        order = np.argsort(np.linalg.norm(P - np.array(v.pos), axis=1), kind="stable")
        for i in range(len(X)):
            per = [o.trace_one_probe(int(p), X[i], D[i], 0.0, np.inf)[0] for p in order]
            hits = [q for q, c in enumerate(per) if c == oracle.HIT]
            if hits:
                assert res["cls"][i] == oracle.HIT and res["probe"][i] == order[hits[0]]
                n_fell_through += hits[0] > 0
            else:
                want = oracle.UNKNOWN if oracle.UNKNOWN in per else oracle.MISS
                assert res["cls"][i] == want and res["probe"][i] == -1
    assert n_fell_through > 0  # the fall-through path was exercised


def test_nearest_mode_hits_agree_with_analytic_truth():
    """The four-probe workload: where the true hit T is visible from the HIT
    probe, the HIT texel is within one texel of oct(T - O) (regression floor,
    silhouettes excepted as in the grid mode)."""
    sc, views = synth.workload("few")
    d, n, r = sc.probe_maps()
    v = views[0]
    pix = np.arange(0, v.W * v.H, 97)
    res = oracle.Oracle(sc.grid, d, n, r, traversal=1).render(v, pix)
    hit = res["cls"] == oracle.HIT
    assert hit.mean() > 0.6
    X, D = camera_rays(v, pix)
    t, _, _, _ = sc.cast(X, D)
    T = (X + t[:, None] * D)[hit]
    O = sc.grid.probe_positions()[res["probe"][hit]]
    dirs = T - O
    dd = np.linalg.norm(dirs, axis=1)
    tv, _, _, _ = sc.cast(O, dirs / dd[:, None])
    visible = np.abs(tv - dd) < 1e-6 * np.maximum(1.0, dd)
    p = oracle.oct_encode(dirs)
    want = np.clip(np.floor((p + 1) / 2 * sc.grid.N).astype(int), 0, sc.grid.N - 1)
    assert _within_one_texel(sc.grid.N, res["texel"][hit][visible], want[visible]).mean() >= 0.95


def test_eye_nearest_lookup_returns_the_texel_holding_oct_w(tiny):
    """Eye at a probe with the texel fetch: rgb is exactly the stored radiance
    of the texel that contains oct(w), and that texel's centre direction lies
    within a texel's angular size of w; bilinear mode differs off-centre."""
    sc, views, d, n, r = tiny
    g = sc.grid
    P = g.probe_positions()
    rng = np.random.default_rng(5)
    W = rng.normal(size=(2000, 3))
    W /= np.linalg.norm(W, axis=1, keepdims=True)
    near = oracle.Oracle(g, d, n, r, eye_nearest=True)
    bil = oracle.Oracle(g, d, n, r)
    dirs = synth.texel_directions(g.N)
    for probe in (0, 6):
        X = np.repeat(P[probe][None], len(W), 0)
        a = near.trace_rays(X, W)
        b = bil.trace_rays(X, W)
        assert np.all(a["cls"] == oracle.HIT) and np.all(a["probe"] == probe)
        i, j = a["texel"][:, 0], a["texel"][:, 1]
        p = oracle.oct_encode(W)
        assert np.array_equal(i, np.clip(np.floor((p[:, 0] + 1) / 2 * g.N), 0, g.N - 1).astype(int))
        assert np.array_equal(j, np.clip(np.floor((p[:, 1] + 1) / 2 * g.N), 0, g.N - 1).astype(int))
        np.testing.assert_allclose(a["rgb"], r[probe, j, i], atol=1e-12, rtol=0)
        ang = np.arccos(np.clip(np.sum(dirs[j, i] * W, axis=1), -1, 1))
        assert ang.max() < 4.5 / g.N  # centre-to-corner angle of a texel: sup ~4.21 / N
        assert np.abs(a["rgb"] - b["rgb"]).max() > 1e-3


def test_incoming_normal_plane_points_from_the_surface_to_the_probe(tiny):
    """normal_mode='incoming': each texel stores minus its own direction; the
    encoder maps minus the stored vector back into the same texel."""
    sc, views, d, n, r = tiny
    N = sc.grid.N
    d2, n2, r2 = sc.probe_maps(normal_mode="incoming")
    assert np.array_equal(d, d2) and np.array_equal(r, r2)
    np.testing.assert_allclose(np.linalg.norm(n2, axis=-1), 1.0, atol=1e-6)
    p = oracle.oct_encode(-n2[3].reshape(-1, 3).astype(np.float64))
    ij = np.clip(np.floor((p + 1) / 2 * N).astype(int), 0, N - 1)
    jj, ii = np.divmod(np.arange(N * N), N)
    assert np.array_equal(ij[:, 0], ii) and np.array_equal(ij[:, 1], jj)


@pytest.mark.parametrize("N,M,dims,spacing", [(64, 16, (2, 2, 2), 1.0), (128, 16, (3, 3, 3), 0.5)])
def test_incoming_normals_in_an_empty_room_equal_surface_normals(N, M, dims, spacing):
    """Inside a closed convex room every crossing is the ray leaving the probe
    through the wall, so the incoming-direction test accepts exactly what the
    surface-normal test accepts: identical images."""
    g = synth.Grid(*dims, spacing, N, M)
    sc = synth.make_scene(g, 0, 0, [1.0], seed=7)
    v = synth.random_view(sc, 107, 64, 64, 60.0)
    a = oracle.Oracle(g, *sc.probe_maps()).render(v)
    b = oracle.Oracle(g, *sc.probe_maps(normal_mode="incoming")).render(v)
    assert np.all(a["cls"] == oracle.HIT)
    for k in ("cls", "probe", "texel", "rgb"):
        assert np.array_equal(a[k], b[k]), k


def test_incoming_normals_hit_only_where_the_ray_leaves_the_probe(tiny):
    """With incoming-direction normals the normal test of Appendix A
    highResolutionTracing reads 'the ray moves away from the probe at the
    crossing': every HIT ray has w . dir(hit texel) > 0 (synth's texel
    directions), and the cluttered tiny scene stays >= 99 % HIT."""
    sc, views, d, n, r = tiny
    dn, nn, rn = sc.probe_maps(normal_mode="incoming")
    v = views[0]
    res = oracle.Oracle(sc.grid, dn, nn, rn).render(v)
    hit = res["cls"] == oracle.HIT
    assert hit.mean() >= 0.99
    _, D = camera_rays(v)
    dirs = synth.texel_directions(sc.grid.N)
    i, j = res["texel"][hit, 0], res["texel"][hit, 1]
    assert np.all(np.sum(dirs[j, i] * D[hit], axis=1) > 0)
