import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


_CACHE = {}


def load_workload(name):
    """(scene, views, dist, normal, radiance) for a named synthetic workload, cached per session."""
    if name not in _CACHE:
        import synth
        sc, views = synth.workload(name)
        d, n, r = sc.probe_maps()
        _CACHE[name] = (sc, views, d, n, r)
    return _CACHE[name]


def camera_rays(view, pixels=None):
    """Pinhole rays of a view in float64 (ray (X, w1) of Sec. 3), for ground-truth casts."""
    import math
    n = view.W * view.H
    pix = np.arange(n) if pixels is None else np.asarray(pixels)
    xs, ys = pix % view.W, pix // view.W
    th = math.tan(view.fov_y / 2)
    a = ((xs + 0.5) / view.W * 2 - 1) * th * view.W / view.H
    b = (1 - (ys + 0.5) / view.H * 2) * th
    D = (np.array(view.fwd)[None] + a[:, None] * np.array(view.right)[None]
         + b[:, None] * np.array(view.up)[None])
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    X = np.repeat(np.array(view.pos, dtype=np.float64)[None], len(D), 0)
    return X, D


@pytest.fixture(scope="session")
def tiny():
    return load_workload("tiny")


@pytest.fixture(scope="session")
def room():
    return load_workload("room")
