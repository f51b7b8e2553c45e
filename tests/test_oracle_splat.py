"""Pins for the oracle's point-cloud probe builder (Sec. 4.1 simulated probe
data, Sec. 5.1 probe data generation): nearest point per texel, from clouds
with closed-form answers, brute force, and the analytic scene."""
import numpy as np
import pytest

import oracle
import synth
from conftest import camera_rays


def _fib_sphere(n, centre, R):
    k = np.arange(n)
    z = 1 - (2 * k + 1) / n
    r = np.sqrt(1 - z * z)
    phi = k * np.pi * (3 - np.sqrt(5))
    return (np.asarray(centre) + R * np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)).astype(np.float32)


def test_sphere_shell_gives_its_radius_everywhere():
    """A dense shell of radius R around the probe fills every texel with
    distance R (float32 rounding), its colour, and incoming directions within
    a texel's angle of minus the texel direction."""
    N, R = 32, 0.7
    O = np.array([[0.1, 0.2, 0.3]], np.float32)
    xyz = _fib_sphere(400000, O[0], R)
    rgb = np.tile(np.float32([[0.2, 0.4, 0.6]]), (len(xyz), 1))
    d, n, r = oracle.splat_probes(xyz, rgb, O, N)
    assert np.abs(d - R).max() <= 2e-6 * R
    assert np.array_equal(r[0], np.broadcast_to(np.float32([0.2, 0.4, 0.6]), (N, N, 3)))
    ang = np.arccos(np.clip(np.sum(-n[0] * synth.texel_directions(N), -1), -1, 1))
    assert ang.max() < 4.5 / N
    np.testing.assert_allclose(np.linalg.norm(n, axis=-1), 1.0, atol=1e-6)


def test_nearer_shell_occludes_the_farther_one_and_holes_stay_empty():
    """Two shells: the inner one wins every texel (distance and colour). A
    hemisphere (z >= 0 in the probe frame) leaves the lower texels empty:
    distance empty_dist, radiance 0, normal minus the texel direction."""
    N = 16
    O = np.zeros((1, 3), np.float32)
    a, b = _fib_sphere(100000, O[0], 2.0), _fib_sphere(100000, O[0], 0.5)
    xyz = np.concatenate([a, b])
    rgb = np.concatenate([np.tile(np.float32([[1, 0, 0]]), (len(a), 1)), np.tile(np.float32([[0, 0, 1]]), (len(b), 1))])
    d, n, r = oracle.splat_probes(xyz, rgb, O, N)
    assert np.abs(d - 0.5).max() <= 1e-6 and np.all(r[..., 2] == 1) and np.all(r[..., 0] == 0)
    upper = b[b[:, 2] >= 0.05]
    d, n, r = oracle.splat_probes(upper, np.ones_like(upper), O, N, empty_dist=-1.0)
    dirs = synth.texel_directions(N)
    lower = dirs[..., 2] < -0.2  # texels whose whole footprint is below the cap
    assert np.all(d[0][lower] == -1.0) and np.all(r[0][lower] == 0)
    np.testing.assert_allclose(n[0][lower], -dirs[lower], atol=1e-6)
    assert np.all(d[0][dirs[..., 2] > 0.3] > 0)


def test_brute_force_nearest_point_per_texel_with_ties():
    """Tiny cloud, every texel's winner found by a Python loop over points
    (float32 binning as the builder states it); duplicated points make exact
    ties, which the lower point index wins."""
    rng = np.random.default_rng(4)
    N = 4
    pts = rng.uniform(-1, 1, (300, 3)).astype(np.float32)
    pts = np.concatenate([pts, pts[:40]])  # indices 300.. duplicate 0..39
    rgb = rng.uniform(0, 1, (len(pts), 3)).astype(np.float32)
    probes = np.float32([[0.05, -0.1, 0.2], [0.3, 0.3, -0.4]])
    d, n, r = oracle.splat_probes(pts, rgb, probes, N, empty_dist=-1.0)
    f = np.float32
    for p, O in enumerate(probes):
        best = {}
        for k, x in enumerate(pts):
            v = x - O
            q = f(f(v[0] * v[0]) + f(v[1] * v[1]))
            q = f(q + f(v[2] * v[2]))
            s = f(f(abs(v[0]) + abs(v[1])) + abs(v[2]))
            inv = f(f(1) / s)
            px, py = f(v[0] * inv), f(v[1] * inv)
            if v[2] < 0:
                px, py = (f((f(1) - abs(py)) * (1 if px >= 0 else -1)), f((f(1) - abs(px)) * (1 if py >= 0 else -1)))
            i = min(max(int(np.floor(f((px + f(1)) * f(N / 2)))), 0), N - 1)
            j = min(max(int(np.floor(f((py + f(1)) * f(N / 2)))), 0), N - 1)
            if (j, i) not in best or (q, k) < best[(j, i)]:
                best[(j, i)] = (q, k)
        for j in range(N):
            for i in range(N):
                if (j, i) in best:
                    q, k = best[(j, i)]
                    assert k < 300
                    assert d[p, j, i] == np.sqrt(q) and np.array_equal(r[p, j, i], rgb[k])
                else:
                    assert d[p, j, i] == -1.0


@pytest.fixture(scope="module")
def scanned_tiny():
    sc, views = synth.workload("tiny")
    pc = synth.scan(sc, synth.scan_positions(sc, 4, 77), 1000000, seed=9)
    maps = oracle.splat_probes(pc["xyz"], pc["rgb"], sc.grid.probe_positions(), sc.grid.N)
    return sc, views, pc, maps


def test_splatted_winners_are_the_surfaces_the_probe_sees(scanned_tiny):
    """Four simulated scans of the tiny scene: a texel's winner is a surface
    point, so the analytic cast from the probe towards it never goes past it,
    and for >= 99 % of texels it stops at it (the probe sees the winner)."""
    sc, views, pc, (d, n, r) = scanned_tiny
    filled = d > 0
    assert filled.mean() > 0.95
    P = sc.grid.probe_positions()
    pid = np.repeat(np.arange(len(P)), sc.grid.N ** 2).reshape(d.shape)[filled]
    w = -n[filled].astype(np.float64)
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    t, _, _, _ = sc.cast(P[pid], w)
    assert np.all(t <= d[filled] * (1 + 1e-5))
    assert (np.abs(t - d[filled]) <= 1e-5 * d[filled]).mean() >= 0.99


def test_render_from_scanned_probes(scanned_tiny):
    """The paper's pipeline end to end (scan -> probe maps -> trace): the
    image from splatted probes is almost all HIT and close to the analytic
    radiance for a large share of pixels (regression floors; ray-cast probes
    reach 61 % within 0.05 on this view, splatted ones 40 %: the nearest point
    of a texel is not at its centre)."""
    sc, views, pc, maps = scanned_tiny
    v = views[0]
    res = oracle.Oracle(sc.grid, *maps).render(v)
    X, D = camera_rays(v)
    _, _, truth, _ = sc.cast(X, D)
    hit = res["cls"] == oracle.HIT
    assert hit.mean() >= 0.99
    assert ((np.abs(res["rgb"] - truth).max(1) < 0.05) & hit).mean() >= 0.35
