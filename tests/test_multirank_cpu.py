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
