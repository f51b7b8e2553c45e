"""Pins for the oracle's adjoint. For fixed distance and normal maps the hit
texel and bilinear weights do not depend on radiance, so the rendered colour is
linear in the radiance maps (Sec. 3: L_o(X, w1) = L_p(w2), looked up
bilinearly); the adjoint scatters each pixel's gradient through those weights."""
import numpy as np
import pytest

import oracle
import synth


def sub_instance():
    """2x2x2 cage, 32x32 maps, 8x8 mip, one 48x48 view (seeded like the tiny workload)."""
    g = synth.Grid(2, 2, 2, 1.0, 32, 8)
    sc = synth.make_scene(g, 8, 2, [1.0], seed=1)
    v = synth.random_view(sc, 101, 48, 48, 60.0)
    d, n, r = sc.probe_maps()
    return g, sc, v, d, n, r


@pytest.fixture(scope="module")
def inst():
    return sub_instance()


def test_adjoint_identity(inst):
    """<g, A rad> == <A^T g, rad> for random g (A = render as a linear map of radiance)."""
    g, sc, v, d, n, r = inst
    o = oracle.Oracle(g, d, n, r)
    out = o.render(v)
    rng = np.random.default_rng(1)
    gr = rng.normal(size=out["rgb"].shape)
    grad = o.backward(gr, out["cls"], out["probe"], out["uv"])
    lhs = float((gr * out["rgb"]).sum())
    rhs = float((grad * r.astype(np.float64)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_adjoint_matches_central_differences(inst):
    g, sc, v, d, n, r = inst
    o = oracle.Oracle(g, d, n, r)
    out = o.render(v)
    rng = np.random.default_rng(2)
    gr = rng.normal(size=out["rgb"].shape)
    grad = o.backward(gr, out["cls"], out["probe"], out["uv"])
    used = np.argwhere(np.abs(grad) > 1e-3)
    assert len(used) > 50
    pick = used[rng.choice(len(used), 40, replace=False)]
    h = 0.125  # linear map: the difference quotient is exact up to rounding for any step
    for p, j, i, c in pick:
        rp = r.copy()
        rm = r.copy()
        rp[p, j, i, c] += h
        rm[p, j, i, c] -= h
        fp = oracle.Oracle(g, d, n, rp).render(v)["rgb"]
        fm = oracle.Oracle(g, d, n, rm).render(v)["rgb"]
        fd = float((gr * (fp - fm)).sum()) / (float(rp[p, j, i, c]) - float(rm[p, j, i, c]))
        assert abs(fd - grad[p, j, i, c]) <= 1e-9 * max(1.0, abs(grad[p, j, i, c]))


def test_geometry_does_not_depend_on_radiance(inst):
    """Class, probe and hit texel are unchanged when radiance is replaced."""
    g, sc, v, d, n, r = inst
    a = oracle.Oracle(g, d, n, r).render(v)
    r2 = np.random.default_rng(3).uniform(0, 1, r.shape).astype(np.float32)
    b = oracle.Oracle(g, d, n, r2).render(v)
    for k in ("cls", "probe", "texel", "uv", "t_hit"):
        assert np.array_equal(a[k], b[k])
