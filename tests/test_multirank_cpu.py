"""The multi-rank bench path on CPU: two gloo ranks (weak scaling, no
data-path collective; only the timing is reduced across ranks)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (r + 1) seconds for 1e6 * (r + 1) rays
    value, seconds, rays = bench.aggregate_over_ranks(float(rank + 1), 1e6 * (rank + 1))
    q.put((rank, value, seconds, rays, bench.dist_env()))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_all_rays():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, seconds, rays, env in res:
        assert seconds == 2.0 and rays == 3e6
        assert value == pytest.approx(3e6 / 2.0 / 1e6)
        assert env[0] == rank and env[1] == 2


def test_single_process_value_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, seconds, rays = bench.aggregate_over_ranks(0.5, 2e6)
    assert value == pytest.approx(4.0) and seconds == 0.5 and rays == 2e6


def _fit_rank(rank, world, port, q):
    """One rank of the data-parallel fit step on CPU: its shard of the views,
    the oracle's adjoint of its pixels, then the gradient all-reduce."""
    import numpy as np
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    from paper_2507_14624_gb300 import fit  # host helpers only; no GPU call
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = synth.Grid(2, 2, 2, 1.0, 32, 8)
    sc = synth.make_scene(g, 8, 2, [1.0], seed=1)
    d, n, r = sc.probe_maps()
    o = oracle.Oracle(g, d, n, r)
    views = [synth.random_view(sc, 300 + k, 24 + 4 * k, 20, 60.0) for k in range(5)]
    rng = np.random.default_rng(0)
    grad_rgb = [rng.normal(size=(v.W * v.H, 3)) for v in views]  # same on every rank
    mine = fit.shard_views(views, rank, world)
    idx = fit.shard_pixels(views, rank, world)
    grad = np.zeros((8, 32, 32, 3))
    for v, (b, e) in zip(mine, idx):
        out = o.render(v)
        k = views.index(v)
        assert e - b == v.W * v.H
        grad += o.backward(grad_rgb[k], out["cls"], out["probe"], out["uv"])
    t = torch.tensor(grad)
    fit.allreduce_gradient(t)
    q.put((rank, t.numpy(), [views.index(v) for v in mine]))
    dist.destroy_process_group()


def test_data_parallel_fit_gradient_equals_the_single_process_gradient():
    """Two gloo ranks each take every other view and the oracle's adjoint of
    their pixels; after the all-reduce both hold the gradient of all views."""
    import multiprocessing as mp
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_fit_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][2] == [0, 2, 4] and res[1][2] == [1, 3]
    g = synth.Grid(2, 2, 2, 1.0, 32, 8)
    sc = synth.make_scene(g, 8, 2, [1.0], seed=1)
    d, n, r = sc.probe_maps()
    o = oracle.Oracle(g, d, n, r)
    views = [synth.random_view(sc, 300 + k, 24 + 4 * k, 20, 60.0) for k in range(5)]
    rng = np.random.default_rng(0)
    full = np.zeros((8, 32, 32, 3))
    for v in views:
        gr = rng.normal(size=(v.W * v.H, 3))
        out = o.render(v)
        full += o.backward(gr, out["cls"], out["probe"], out["uv"])
    for rank, grad, _ in res:
        np.testing.assert_allclose(grad, full, rtol=0, atol=1e-9 * max(1.0, np.abs(full).max()))
