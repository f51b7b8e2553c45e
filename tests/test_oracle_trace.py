"""Pins for the oracle's tracer: Appendix A algorithms, Sec. 4.2-4.3, against
the analytic scene, brute force and invariants the method fixes."""
import numpy as np
import pytest

import oracle
import synth
from conftest import camera_rays


def _within_one_texel(N, got, want):
    """Mirror-aware Chebyshev distance <= 1 between texel (i, j) pairs."""
    ok = np.zeros(len(got), bool)
    for k, ((gi, gj), (wi, wj)) in enumerate(zip(got, want)):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                if oracle.mirror_texel(N, int(gi) + di, int(gj) + dj) == (int(wi), int(wj)):
                    ok[k] = True
    return ok


def test_mip_is_conservative_exhaustive(tiny):
    sc, views, d, n, r = tiny
    N, M = sc.grid.N, sc.grid.M
    mn, mx = oracle.build_mip(d, M)
    k = N // M
    blocks = d.reshape(d.shape[0], M, k, M, k)
    assert np.array_equal(mn, blocks.min(axis=(2, 4)))
    assert np.array_equal(mx, blocks.max(axis=(2, 4)))
    # every fine texel lies within its coarse [min, max]
    up_mn = np.repeat(np.repeat(mn, k, 1), k, 2)
    up_mx = np.repeat(np.repeat(mx, k, 1), k, 2)
    assert np.all(up_mn <= d) and np.all(d <= up_mx)


@pytest.mark.parametrize("name,stride", [("tiny", 1), ("room", 11)])
def test_hierarchical_march_equals_flat_march(name, stride, request):
    """Low-resolution tracing only skips what the full-resolution march would
    pass (min/max mip), so class and hit texel agree on every pixel."""
    sc, views, d, n, r = request.getfixturevalue(name)
    v = views[0]
    o = oracle.Oracle(sc.grid, d, n, r)
    pix = np.arange(0, v.W * v.H, stride)
    flat = o.render(v, pix, march=oracle.MARCH_FLAT)
    for mode in (oracle.MARCH_HIER, oracle.MARCH_HIER_SHORTCUT):
        h = o.render(v, pix, march=mode)
        assert np.array_equal(h["cls"], flat["cls"])
        assert np.array_equal(h["probe"], flat["probe"])
        assert np.array_equal(h["texel"], flat["texel"])
        assert np.array_equal(h["rgb"], flat["rgb"])


@pytest.mark.parametrize("N,M,dims,spacing", [(64, 16, (2, 2, 2), 1.0), (128, 16, (3, 3, 3), 0.5),
                                              (32, 8, (2, 2, 2), 1.0)])
def test_empty_room_is_exact(N, M, dims, spacing):
    """A closed convex room seen from inside has no silhouettes, so every probe
    sees the true hit T (Sec. 3: visible iff r_p(w2) = d(O, T)): every pixel is
    a HIT whose texel is within one texel of oct(T - O)."""
    g = synth.Grid(*dims, spacing, N, M)
    sc = synth.make_scene(g, 0, 0, [1.0], seed=7)
    v = synth.random_view(sc, 107, 96, 96, 60.0)
    d, n, r = sc.probe_maps()
    res = oracle.Oracle(g, d, n, r).render(v)
    assert np.all(res["cls"] == oracle.HIT)
    X, D = camera_rays(v)
    t, _, rgb, _ = sc.cast(X, D)
    T = X + t[:, None] * D
    O = g.probe_positions()[res["probe"]]
    p = oracle.oct_encode(T - O)
    want = np.clip(np.floor((p + 1) / 2 * N).astype(int), 0, N - 1)
    assert np.all(_within_one_texel(N, res["texel"], want))
    # the hit point is on the wall within a texel footprint
    assert np.max(np.abs(res["t_hit"] - t) / t) < 8.0 / N


@pytest.mark.parametrize("name,stride,floor", [("tiny", 1, 0.95), ("room", 23, 0.95)])
def test_cluttered_scene_hits_agree_with_analytic_truth(name, stride, floor, request):
    """Where the true hit T is visible from the probe that returned HIT, the HIT
    texel is within one texel of oct(T - O) for all but the silhouette cases
    (a texel that straddles an object's outline stores the object's depth, and
    a ray grazing past the outline crosses it: the resolution artefact of
    Sec. 6, 'jig jags'). The fraction is a regression floor."""
    sc, views, d, n, r = request.getfixturevalue(name)
    v = views[0]
    pix = np.arange(0, v.W * v.H, stride)
    res = oracle.Oracle(sc.grid, d, n, r).render(v, pix)
    X, D = camera_rays(v, pix)
    t, _, _, _ = sc.cast(X, D)
    T = X + t[:, None] * D
    hit = res["cls"] == oracle.HIT
    assert hit.mean() > 0.8
    O = sc.grid.probe_positions()[res["probe"][hit]]
    dirs = T[hit] - O
    dd = np.linalg.norm(dirs, axis=1)
    tv, _, _, _ = sc.cast(O, dirs / dd[:, None])
    visible = np.abs(tv - dd) < 1e-6 * np.maximum(1.0, dd)
    p = oracle.oct_encode(dirs)
    N = sc.grid.N
    want = np.clip(np.floor((p + 1) / 2 * N).astype(int), 0, N - 1)
    ok = _within_one_texel(N, res["texel"][hit][visible], want[visible])
    assert ok.mean() >= floor


def test_eye_aligned_lookup_at_texel_centres(tiny):
    """Eye at a probe (Appendix A traceOneProbe, X == probeOrigin): rays along
    texel-centre directions return exactly the stored radiance of that texel,
    and every ray is a HIT (closed room)."""
    sc, views, d, n, r = tiny
    g = sc.grid
    o = oracle.Oracle(g, d, n, r)
    P = g.probe_positions()
    dirs = synth.texel_directions(g.N)
    rng = np.random.default_rng(3)
    for probe in (0, 5, 7):
        jj = rng.integers(0, g.N, 400)
        ii = rng.integers(0, g.N, 400)
        W = dirs[jj, ii]
        X = np.repeat(P[probe][None], len(W), 0)
        res = o.trace_rays(X, W)
        assert np.all(res["cls"] == oracle.HIT)
        assert np.all(res["probe"] == probe)
        np.testing.assert_allclose(res["rgb"], r[probe, jj, ii], atol=1e-6, rtol=0)
        assert np.array_equal(res["texel"], np.stack([ii, jj], 1))


def test_closed_room_has_no_miss(tiny, room):
    """The last cell extends to infinity and the room is closed, so the ray's
    radial distance eventually exceeds every stored distance: no pixel is MISS."""
    for sc, views, d, n, r in (tiny, room):
        v = views[0]
        pix = np.arange(0, v.W * v.H, 1 if v.W * v.H < 20000 else 29)
        res = oracle.Oracle(sc.grid, d, n, r).render(v, pix)
        assert not np.any(res["cls"] == oracle.MISS)


def test_grid_iterator_brute_force(room):
    """Cells come in ray order, tile [0, inf), and each cell's interval is the
    part of the ray inside that cell (brute-force point location)."""
    sc, views, d, n, r = room
    o = oracle.Oracle(sc.grid, d, n, r)
    g = sc.grid
    rng = np.random.default_rng(9)
    for _ in range(300):
        X = g.lo() + rng.uniform(0.05, 0.95, 3) * (g.hi() - g.lo())
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        cells = o.grid_cells(X, w)
        assert cells[0][1] == 0.0 and np.isinf(cells[-1][2])
        for (c0, a0, b0), (c1, a1, b1) in zip(cells[:-1], cells[1:]):
            assert b0 == a1 and a0 < b0
            assert sum(abs(x - y) for x, y in zip(c0, c1)) == 1
        for c, a, b in cells:
            tm = 0.5 * (a + b) if np.isfinite(b) else a + 1e-9
            pnt = X + tm * w
            cell = np.floor((pnt - g.lo()) / g.spacing).astype(int)
            cell = np.clip(cell, 0, np.array([g.nx, g.ny, g.nz]) - 2)
            assert tuple(cell) == tuple(c)


def test_cage_order_is_nearest_first(room):
    sc, views, d, n, r = room
    o = oracle.Oracle(sc.grid, d, n, r)
    P = sc.grid.probe_positions()
    rng = np.random.default_rng(10)
    for _ in range(200):
        c = rng.integers(0, 3, 3)
        pt = sc.grid.lo() + (c + rng.uniform(0, 1, 3)) * sc.grid.spacing
        order = o.cage_order(c, pt)
        dist = np.linalg.norm(P[order] - pt, axis=1)
        assert np.all(np.diff(dist) >= 0)
        assert sorted(order) == sorted(
            int(c[0] + dx + 4 * (c[1] + dy + 4 * (c[2] + dz))) for dx in (0, 1) for dy in (0, 1) for dz in (0, 1))


def test_trace_one_probe_in_an_empty_cube_room():
    """Closed form first: a probe at the centre of an empty cube room of
    half-size h stores the distance h / max|u_i| along direction u. Then, with
    probes on the grid, traceOneProbe over [0, inf) from any point inside the
    room is a HIT within one texel of the analytic wall hit."""
    g = synth.Grid(2, 2, 2, 1.0, 128, 16)
    sc = synth.make_scene(g, 0, 0, [1.0], seed=8)
    centre = 0.5 * (g.lo() + g.hi())
    d, _, _ = sc.probe_maps(probe_pos=centre[None])
    dirs = synth.texel_directions(g.N)
    h = 0.5 * (sc.room[3] - sc.room[0])
    np.testing.assert_allclose(d[0], h / np.abs(dirs).max(-1), rtol=1e-6)

    # With the listing's two-way rule (every crossing goes to the normal test)
    # each single-probe trace is a HIT on the inward-facing wall; with the
    # passes-behind branch a grazing wall can give UNKNOWN (the texel-centre
    # depth jumps by more than the thickness), never MISS.
    d2, n2, r2 = sc.probe_maps()
    P = g.probe_positions()
    for th_rel in (-1.0, 1.0):
        o = oracle.Oracle(g, d2, n2, r2, thickness_rel=th_rel)
        rng = np.random.default_rng(12)
        n_hit = 0
        for _ in range(300):
            X = g.lo() + rng.uniform(0.1, 0.9, 3) * (g.hi() - g.lo())
            w = rng.normal(size=3)
            w /= np.linalg.norm(w)
            probe = int(rng.integers(0, 8))
            cls, tex, uv, th = o.trace_one_probe(probe, X, w, 0.0, np.inf)
            assert cls != oracle.MISS
            if th_rel < 0:
                assert cls == oracle.HIT
            if cls != oracle.HIT:
                continue
            n_hit += 1
            t, _, _, _ = sc.cast(X[None], w[None])
            T = X + t[0] * w
            p = oracle.oct_encode(T - P[probe])
            want = np.clip(np.floor((p + 1) / 2 * g.N).astype(int), 0, g.N - 1)
            assert _within_one_texel(g.N, [tex], [want])[0]
        assert n_hit >= 250


def _sphere_maps(g, R, w):
    """Every probe stores distance R in every texel (a sphere of radius R
    around it) and the normal -w for one ray direction w, so a crossing by a
    ray along w always passes the normal test."""
    P, N = g.n_probes, g.N
    d = np.full((P, N, N), R, np.float32)
    n = np.broadcast_to(-np.asarray(w, np.float32), (P, N, N, 3)).copy()
    r = np.zeros((P, N, N, 3), np.float32)
    return d, n, r


def _roots(Y0, w, R):
    """Both roots of |Y0 + t w| = R (|w| = 1), in the cancellation-free forms."""
    B = float(np.dot(Y0, w))
    C = float(np.dot(Y0, Y0)) - R * R
    disc = B * B - C
    s = np.sqrt(max(disc, 0.0))
    if B > 0:
        q = -(B + s)
        return C / q, q
    q = s - B
    return C / q if q != 0 else -B, q


@pytest.mark.parametrize("case", ["in_front", "behind_approaching", "behind_receding", "never_reaches"])
def test_hit_point_is_the_analytic_root(case):
    """Hit point inside the deciding texel (the reading of the paper's
    highResolutionTracing, which returns only the texel): against a probe
    whose map holds a sphere of radius R, traceOneProbe returns
      - a ray starting inside the sphere: the larger root of |X + t w - O| = R;
      - starting just outside and approaching: the smaller root;
      - starting just outside and receding: the segment start t = 0;
      - approaching but passing the probe at more than R: the closest
        approach -(X - O).w.
    Closed forms to 1e-9; exchanging the two roots fails the first two cases."""
    g = synth.Grid(2, 2, 2, 1.0, 64, 16)
    R = 0.375
    O = g.probe_positions()[5]
    rng = np.random.default_rng({"in_front": 1, "behind_approaching": 2, "behind_receding": 3,
                                 "never_reaches": 4}[case])
    for _ in range(40):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        v = rng.normal(size=3)
        v -= np.dot(v, u) * u
        v /= np.linalg.norm(v)
        if case == "in_front":
            Y0 = rng.uniform(0.05, 0.9) * R * u
            w = rng.normal(size=3)
        elif case == "behind_approaching":
            Y0 = R * (1 + 1e-3) * u
            w = -u + rng.uniform(-0.3, 0.3) * v  # mostly towards the probe: reaches R at once
        elif case == "behind_receding":
            Y0 = R * (1 + 1e-3) * u
            w = u + rng.uniform(-0.5, 0.5) * v
        else:
            Y0 = R * (1 + 1e-2) * u
            w = v - 1e-4 * u  # nearly tangent, approaching: closest approach just above R
        w = w / np.linalg.norm(w)
        X = O + Y0
        d, n, r = _sphere_maps(g, R, w)
        o = oracle.Oracle(g, d, n, r)
        cls, tex, uv, th = o.trace_one_probe(5, X, w, 0.0, np.inf)
        assert cls == oracle.HIT
        small, large = sorted(_roots(Y0, w, R))
        B = float(np.dot(Y0, w))
        if case == "in_front":
            want = large
        elif case == "behind_approaching":
            assert B * B - (np.dot(Y0, Y0) - R * R) > 0
            want = small
        elif case == "behind_receding":
            assert B > 0
            want = 0.0
        else:
            assert B * B - (np.dot(Y0, Y0) - R * R) < 0 and B < 0
            want = -B
        assert abs(th - want) <= 1e-9, (case, th, want)
        if case != "behind_receding":  # the point found lies on the ray at the expected radius
            rad = np.linalg.norm(Y0 + th * w)
            assert abs(rad - (R if case != "never_reaches" else np.sqrt(np.dot(Y0, Y0) - B * B))) <= 1e-9


@pytest.mark.parametrize("N,M", [(48, 16), (96, 8), (192, 16), (192, 8), (144, 6), (192, 4)])
def test_hierarchical_march_equals_flat_march_at_odd_block_sizes(N, M):
    """The min/max skip is exact for any block side k = N / M, including the
    non-powers of two of the resolution study (k = 3, 12, 24, 48 here): class,
    probe, hit texel and radiance agree with the flat march on every pixel."""
    g = synth.Grid(3, 3, 2, 0.5, N, M)
    sc = synth.make_scene(g, 12, 4, [0.7, 0.3], seed=N + M)
    v = synth.random_view(sc, 300 + N, 64, 48, 70.0)
    d, n, r = sc.probe_maps()
    o = oracle.Oracle(g, d, n, r)
    flat = o.render(v, march=oracle.MARCH_FLAT)
    for mode in (oracle.MARCH_HIER, oracle.MARCH_HIER_SHORTCUT):
        h = o.render(v, march=mode)
        for k in ("cls", "probe", "texel", "rgb"):
            assert np.array_equal(h[k], flat[k]), (N, M, k)
    assert (flat["cls"] == oracle.HIT).mean() > 0.8
