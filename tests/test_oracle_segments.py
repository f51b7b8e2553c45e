"""Pins for the octant split and the texel walk along a segment (Sec. 4.2:
projecting the ray onto the octahedral map gives at most 4 segments)."""
import numpy as np

import oracle


def _rand_rays(rng, n):
    X = rng.uniform(-1, 1, size=(n, 3))
    W = rng.normal(size=(n, 3))
    W /= np.linalg.norm(W, axis=1, keepdims=True)
    return X, W


def test_split_gives_at_most_four_single_octant_segments():
    rng = np.random.default_rng(5)
    X, W = _rand_rays(rng, 2000)
    O = np.zeros(3)
    for x, w in zip(X, W):
        segs = oracle.split_segments(x, w, O, 0.0, np.inf)
        assert 1 <= len(segs) <= 4
        for ta, tb in segs:
            # every interior point of a segment has the same octant
            ts = ta + (np.array([0.1, 0.3, 0.5, 0.7, 0.9]) * (tb - ta) if np.isfinite(tb)
                       else np.array([0.01, 0.1, 1, 10, 100]))
            s = np.sign(x[None] + ts[:, None] * w[None])
            assert np.all(s == s[0])


def test_segment_image_is_a_straight_line_and_continuous():
    rng = np.random.default_rng(6)
    X, W = _rand_rays(rng, 2000)
    for x, w in zip(X, W):
        for ta, tb in oracle.split_segments(x, w, np.zeros(3), 0.0, 50.0):
            ts = ta + np.linspace(0.05, 0.95, 5) * (tb - ta)
            p = oracle.oct_encode(x[None] + ts[:, None] * w[None])
            v = p[1:] - p[0]
            cross = v[:, 0] * v[-1, 1] - v[:, 1] * v[-1, 0]
            assert np.max(np.abs(cross)) <= 1e-10
            # continuity inside the segment: the step in p is bounded by a
            # constant times the angle between consecutive directions
            tt = ta + np.linspace(1e-6, 1 - 1e-6, 400) * (tb - ta)
            yy = x[None] + tt[:, None] * w[None]
            yy /= np.linalg.norm(yy, axis=1, keepdims=True)
            pp = oracle.oct_encode(yy)
            ang = np.arccos(np.clip((yy[1:] * yy[:-1]).sum(1), -1, 1))
            assert np.all(np.abs(np.diff(pp, axis=0)).max(1) <= 2.0 * ang + 1e-9)


def test_walk_visits_exactly_the_texels_the_segment_passes_through():
    """Brute force on small maps: dense sampling of the segment in t must see
    the same texels, in the same order, as the DDA walk; intervals tile the segment."""
    rng = np.random.default_rng(7)
    R = 16
    checked = 0
    for _ in range(400):
        x = rng.uniform(-1, 1, 3)
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        for ta, tb in oracle.split_segments(x, w, np.zeros(3), 0.0, 4.0):
            ij, tt = oracle.walk_segment(x, w, ta, tb, R)
            assert len(ij) >= 1
            assert abs(tt[0, 0] - ta) < 1e-12 and abs(tt[-1, 1] - tb) < 1e-12
            assert np.all(np.abs(tt[1:, 0] - tt[:-1, 1]) < 1e-12)
            assert np.all(tt[:, 1] >= tt[:, 0])
            # dense samples, skipping the (measure-zero) boundaries
            ts = np.linspace(ta, tb, 20001)[1:-1]
            p = oracle.oct_encode(x[None] + ts[:, None] * w[None])
            cells = np.clip(np.floor((p + 1) / 2 * R).astype(int), 0, R - 1)
            seq = [tuple(cells[0])]
            for c in map(tuple, cells[1:]):
                if c != seq[-1]:
                    seq.append(c)
            walked = [tuple(c) for c, (a, b) in zip(ij, tt) if b - a > 1e-9 * max(1.0, tb - ta)]
            # sampled sequence must be a subsequence of the walk (tiny texel
            # crossings may fall between samples), and every walked texel of
            # noticeable length must be sampled
            it = iter(walked)
            assert all(any(c == w_ for w_ in it) for c in seq)
            long_ = [tuple(c) for c, (a, b) in zip(ij, tt) if b - a > 1e-3 * (tb - ta)]
            assert set(long_) <= set(seq)
            checked += 1
    assert checked > 400


def test_walk_texel_intervals_contain_their_points():
    rng = np.random.default_rng(8)
    R = 64
    for _ in range(300):
        x = rng.uniform(-1, 1, 3)
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        for ta, tb in oracle.split_segments(x, w, np.zeros(3), 0.0, 10.0):
            ij, tt = oracle.walk_segment(x, w, ta, tb, R)
            mid = 0.5 * (tt[:, 0] + tt[:, 1])
            p = oracle.oct_encode(x[None] + mid[:, None] * w[None])
            cells = np.clip(np.floor((p + 1) / 2 * R).astype(int), 0, R - 1)
            ok = (tt[:, 1] - tt[:, 0]) > 1e-12
            assert np.all(cells[ok] == ij[ok])
