"""Pins for the oracle's multi-scale hierarchy: nested probe grids over the
street-grid scene, each view traced in the finest level whose probe box holds
its camera (the hierarchical representation of the abstract and the teaser
figure)."""
import numpy as np
import pytest

import oracle
import synth
from conftest import camera_rays


@pytest.fixture(scope="module")
def small():
    """The street scene with N and M divided by 8 (L0 N=16, L1 N=32, L2 N=64)."""
    sc, levels, views = synth.multiscale_workload(scale=8, n_views=9)
    maps = [synth.level_scene(sc, g).probe_maps() for g in levels]
    return sc, levels, views, maps


def _inside(g, X):
    """Probe box membership written with the grid's own float32 probe list."""
    P = g.probe_positions()
    return bool(np.all(X >= P.min(0)) and np.all(X <= P.max(0)))


def test_pick_level_is_the_finest_box_holding_the_point(small):
    sc, levels, views, maps = small
    rng = np.random.default_rng(1)
    pts = [rng.uniform(sc.room[:3], sc.room[3:]) for _ in range(3000)]
    for g in levels:  # points on the faces and corners of every box
        P = g.probe_positions()
        lo, hi = P.min(0), P.max(0)
        pts += [lo, hi, np.array([lo[0], hi[1], lo[2]]), 0.5 * (lo + hi)]
        pts += [np.where(rng.random(3) < 0.5, lo, hi) + rng.uniform(-1e-3, 1e-3, 3) for _ in range(200)]
    seen = set()
    for X in pts:
        k = oracle.pick_level(levels, X)
        seen.add(k)
        holding = [j for j, g in enumerate(levels) if _inside(g, X)]
        if holding:
            assert k in holding
            assert all(levels[j].spacing >= levels[k].spacing for j in holding)
        else:
            assert levels[k].spacing == max(g.spacing for g in levels)
    assert seen == {0, 1, 2}


def test_views_cycle_through_the_levels(small):
    sc, levels, views, maps = small
    assert [oracle.pick_level(levels, v.pos) for v in views] == [k % 3 for k in range(len(views))]


def test_finer_levels_are_closer_to_the_analytic_truth():
    """Why the hierarchy exists: for a camera inside a fine level, tracing
    that level gives more HITs and a smaller radiance error against the
    analytic scene than tracing the coarsest level (nearer, denser probes
    and finer maps)."""
    sc, levels, views = synth.multiscale_workload(scale=4, n_views=6)
    maps = [synth.level_scene(sc, g).probe_maps() for g in levels]
    h = oracle.Hierarchy(levels, maps)
    coarse = h.oracles[0]
    for v in views:
        k = h.level_of(v)
        if k == 0:
            continue
        pix = np.arange(0, v.W * v.H, 7)
        X, D = camera_rays(v, pix)
        _, _, truth, _ = sc.cast(X, D)
        fine = h.render(v, pix)
        crs = coarse.render(v, pix)
        assert fine["level"] == k
        assert (fine["cls"] == oracle.HIT).mean() >= (crs["cls"] == oracle.HIT).mean()
        both = (fine["cls"] == oracle.HIT) & (crs["cls"] == oracle.HIT)
        ef = np.abs(fine["rgb"][both] - truth[both]).mean()
        ec = np.abs(crs["rgb"][both] - truth[both]).mean()
        assert ef < ec, (k, ef, ec)


def test_hierarchy_adjoint_identity(small):
    """rgb is linear in each level's radiance: <g, rgb> = sum over levels of
    <grad_l, radiance_l> for the per-level adjoints."""
    sc, levels, views, maps = small
    h = oracle.Hierarchy(levels, maps)
    outs = [h.render(v) for v in views[:6]]
    rgb = np.concatenate([o["rgb"] for o in outs])
    rng = np.random.default_rng(2)
    g = rng.normal(size=rgb.shape)
    grads = h.backward(views[:6], g, np.concatenate([o["cls"] for o in outs]),
                       np.concatenate([o["probe"] for o in outs]), np.concatenate([o["uv"] for o in outs]))
    lhs = float(np.sum(g * rgb))
    rhs = sum(float(np.sum(gr * m[2].astype(np.float64))) for gr, m in zip(grads, maps))
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs))
    assert all(np.abs(gr).sum() > 0 for gr in grads)
