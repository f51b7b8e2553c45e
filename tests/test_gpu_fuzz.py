"""Seeded randomized parity: many small grids and views against the FP64
oracle, through the default (streaming) engine, with the agreement rule of
test_gpu_parity. Each case draws the grid shape (2..4 per axis), spacing,
origin, map sides, thickness rule, texel formats, scene density and camera
(inside or outside the cage, any FOV in 40..110 degrees, odd and even image
sizes). The first set draws powers of two (N in {16..128}, N / M in {2, 4,
8, 16}); the second non-powers of two (N in {48, 96, 192}, block side
k = N / M in {3, 6, 12})."""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import compare

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _case(seed, pow2=True):
    rng = np.random.default_rng(seed)
    dims = tuple(int(x) for x in rng.integers(2, 5, 3))
    spacing = float(rng.choice([0.25, 0.5, 1.0, 1.5]))
    origin = tuple(float(np.float32(x)) for x in rng.uniform(-2, 2, 3))
    if pow2:
        N = int(rng.choice([16, 32, 64, 128]))
        M = N // int(rng.choice([2, 4, 8, 16]))
        M = max(2, M - (M % 2))
    else:  # M = N / k stays even for every pair drawn here
        N = int(rng.choice([48, 96, 192]))
        M = N // int(rng.choice([3, 6, 12]))
    th = float(rng.choice([1.0, 1.0, 0.5, 2.0, -1.0]))
    f16 = bool(rng.random() < 0.3)
    g = synth.Grid(*dims, spacing, N, M, origin)
    sc = synth.make_scene(g, int(rng.integers(0, 40)), int(rng.integers(0, 12)), [0.7, 0.3], seed=seed)
    W, H = int(rng.integers(17, 90)), int(rng.integers(9, 70))
    fov = float(rng.uniform(40, 110))
    if rng.random() < 0.7:
        v = synth.random_view(sc, seed + 17, W, H, fov)
    else:  # anywhere in the room (possibly outside the cage)
        lo, hi = sc.room[:3] + 0.05, sc.room[3:] - 0.05
        while True:
            p = np.float32(rng.uniform(lo, hi)).astype(np.float64)
            if sc.distance_to_objects(p) > 0.03:
                break
        v = synth.look_view(p, rng.uniform(0, 2 * np.pi), rng.uniform(-1.2, 1.2), fov, W, H)
    return g, sc, v, th, f16


@pytest.mark.parametrize("seed,pow2", [(s, True) for s in range(1000, 1024)] +
                         [(s, False) for s in range(2000, 2016)])
def test_random_configuration_matches_oracle(seed, pow2):
    import paper_2507_14624_gb300 as lfpk
    g, sc, v, th, f16 = _case(seed, pow2)
    d, n, r = sc.probe_maps()
    fmt = lfpk.LFP_TEXEL_F16 if f16 else lfpk.LFP_TEXEL_F32
    grid = lfpk.ProbeGrid(g, radiance_fmt=fmt, normal_fmt=fmt, thickness_rel=th)
    grid.upload(d, n, r)
    out = grid.render([v], hit_texel=True)
    ref = oracle.Oracle(g, d, n, r, thickness_rel=th).render(v)
    st = compare(out, ref, g.N)
    # FP16 radiance rounds values <= ~1.1 by <= 4.9e-4; FP16 normals may flip
    # a crossing whose |n . w| is below their octahedral error
    tol_rgb = 1e-3
    tol_dis = max(2e-3 if f16 else 1e-3, 1.0 / v.n_pixels)
    assert st["disagree"] <= tol_dis and st["max_err"] <= tol_rgb, (seed, g, th, f16, st)
    # the loop-nest engine runs the same arithmetic: identical decisions
    b = grid.render([v], hit_texel=True, engine=lfpk.LFP_ENGINE_NESTED)
    for k in ("cls", "probe", "texel"):
        assert torch.equal(out[k], b[k]), (seed, k)
    grid.close()
