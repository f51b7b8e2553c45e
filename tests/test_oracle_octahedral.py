"""Pins for the oracle's octahedral map (Sec. 3, octahedral mapping) and mirror border."""
import os
from fractions import Fraction

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "octahedral_points.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("|")
        d = [float(x) for x in lhs.split()]
        p = [float(Fraction(x)) for x in rhs.split()]
        rows.append((d, p))
    return rows


def test_encode_matches_hand_derived_points():
    rows = _golden()
    assert len(rows) >= 15
    d = np.array([r[0] for r in rows])
    p = np.array([r[1] for r in rows])
    np.testing.assert_allclose(oracle.oct_encode(d), p, atol=1e-15)
    # decode of the golden points gives back the normalised directions
    dn = d / np.linalg.norm(d, axis=1, keepdims=True)
    np.testing.assert_allclose(oracle.oct_decode(p), dn, atol=1e-15)


def test_round_trip_one_million_directions():
    rng = np.random.default_rng(11)
    d = rng.normal(size=(1_000_000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = oracle.oct_encode(d)
    assert np.all(np.abs(p) <= 1.0)
    # the upper hemisphere maps inside the diamond |px| + |py| <= 1
    l1 = np.abs(p).sum(1)
    assert np.all(l1[d[:, 2] > 0] <= 1.0 + 1e-15)
    assert np.all(l1[d[:, 2] < -1e-12] > 1.0 - 1e-12)
    back = oracle.oct_decode(p)
    assert np.max(np.abs(back - d)) <= 1e-12


def test_generator_texel_centres_encode_to_texel_centres():
    """The generator's texel-centre directions (an independent decode) encode
    back to the texel centres: pins the storage convention (i = column / u,
    j = row / v, pole +z) between the two implementations."""
    for N in (8, 64, 256):
        dirs = synth.texel_directions(N)
        p = oracle.oct_encode(dirs)
        jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        want = np.stack([(ii + 0.5) / N * 2 - 1, (jj + 0.5) / N * 2 - 1], axis=-1)
        assert np.max(np.abs(p - want)) <= 1e-12


def _angle(a, b):
    return np.arccos(np.clip((a * b).sum(-1), -1.0, 1.0))


def test_mirror_border_neighbours_are_adjacent_on_the_sphere():
    """Across every edge of the square the mirrored texel is a true neighbour
    on the sphere: within ~1.5 texel pitches of the texel it borders."""
    N = 32
    dirs = synth.texel_directions(N)
    pitch = 4.0 / N  # upper bound on one texel step in radians near the equator
    worst = 0.0
    for k in range(N):
        for (i, j), (bi, bj) in [((-1, k), (0, k)), ((N, k), (N - 1, k)), ((k, -1), (k, 0)), ((k, N), (k, N - 1))]:
            mi, mj = oracle.mirror_texel(N, i, j)
            assert 0 <= mi < N and 0 <= mj < N
            worst = max(worst, float(_angle(dirs[bj, bi], dirs[mj, mi])))
    assert worst <= 1.5 * pitch
    # corners go to the diagonally opposite corner (all four corners are -z)
    assert oracle.mirror_texel(N, -1, -1) == (N - 1, N - 1)
    assert oracle.mirror_texel(N, N, N) == (0, 0)
    assert oracle.mirror_texel(N, N, -1) == (0, N - 1)
    assert oracle.mirror_texel(N, -1, N) == (N - 1, 0)


def test_bilinear_taps_at_texel_centre_are_exact():
    N = 16
    for i, j in [(0, 0), (3, 7), (15, 15), (8, 0)]:
        uv = [(i + 0.5) / N, (j + 0.5) / N]
        ti, tj, w = oracle.bilinear_taps(N, uv)
        k = int(np.argmax(w))
        assert (ti[k], tj[k]) == (i, j) and abs(w[k] - 1.0) < 1e-12
        assert abs(w.sum() - 1.0) < 1e-12


GOLDEN_TAPS = os.path.join(os.path.dirname(__file__), "golden", "bilinear_taps.txt")


def _golden_taps():
    rows = []
    for line in open(GOLDEN_TAPS):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("|")
        N, u, v = lhs.split()
        taps = [tuple(t.split()) for t in rhs.split(";")]
        rows.append((int(N), (float(u), float(v)),
                     [(int(i), int(j), float(w)) for i, j, w in taps]))
    return rows


def test_bilinear_taps_match_hand_derived_table():
    """Taps and weights off texel centres, at the mirror border and past the
    corners, against the table derived by hand in tests/golden/bilinear_taps.txt."""
    rows = _golden_taps()
    assert len(rows) >= 6
    for N, uv, want in rows:
        ti, tj, w = oracle.bilinear_taps(N, uv)
        for k, (i, j, wk) in enumerate(want):
            assert (ti[k], tj[k]) == (i, j), (N, uv, k)
            assert abs(w[k] - wk) <= 1e-15, (N, uv, k)


def test_bilinear_reproduces_affine_maps_off_centre():
    """Bilinear interpolation over texel centres reproduces an affine function
    of the texel coordinate exactly: with c(i, j) = alpha + beta i + gamma j
    stored at the centres, the lookup at uv returns alpha + beta s + gamma t,
    s = u N - 0.5, t = v N - 0.5, wherever all four taps lie inside the map.
    beta != gamma, so exchanging the two fractions, or a weight with its
    complement, moves the result by a multiple of |beta - gamma| or more."""
    rng = np.random.default_rng(21)
    for N in (4, 16, 64):
        alpha, beta, gamma = rng.uniform(-1, 1, 3), rng.uniform(0.5, 2, 3), rng.uniform(-3, -0.5, 3)
        jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        c = alpha + beta * ii[..., None] + gamma * jj[..., None]  # [j][i][3]
        uv = rng.uniform(0.5 / N, (N - 0.5) / N, (400, 2))
        for u, v in uv:
            ti, tj, w = oracle.bilinear_taps(N, (u, v))
            got = (w[:, None] * c[tj, ti]).sum(0)
            want = alpha + beta * (u * N - 0.5) + gamma * (v * N - 0.5)
            assert np.max(np.abs(got - want)) <= 1e-12
            assert abs(w.sum() - 1.0) <= 1e-15 and np.all(w >= 0)
