"""lfp_render_static: the forward render that allocates nothing.

It exists for callers that cannot allocate device memory while they render:
a real-time frame loop that must not touch the allocator after start-up, or a
host whose device memory comes from its own fixed-budget allocator. It keeps
its work-queue head and view table in a fixed file-scope device array, so this
test checks, through the C ABI, that two calls in a row (the second with
different views, so the shared array is reused) give the same images as
lfp_render_ex with the persistent schedule, and that a request beyond the
array's capacity is refused before anything runs.
"""
import ctypes

import numpy as np
import pytest

import synth
from conftest import load_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _outputs(lfp, total, dev):
    t = {"rgb": torch.empty((total, 3), dtype=torch.float32, device=dev),
         "cls": torch.empty(total, dtype=torch.uint8, device=dev),
         "probe": torch.empty(total, dtype=torch.int32, device=dev),
         "uv": torch.empty((total, 2), dtype=torch.float32, device=dev),
         "texel": torch.empty(total, dtype=torch.int32, device=dev)}
    o = lfp.lfp_outputs()
    o.rgb, o.cls, o.aux_probe = t["rgb"].data_ptr(), t["cls"].data_ptr(), t["probe"].data_ptr()
    o.aux_uv, o.hit_texel = t["uv"].data_ptr(), t["texel"].data_ptr()
    return t, o


def test_static_render_matches_persistent_render_twice_in_a_row():
    import paper_2507_14624_gb300 as lfpk
    from paper_2507_14624_gb300 import lfp
    sc, views, d, n, r = load_workload("tiny")
    grid = lfpk.ProbeGrid(sc.grid)
    grid.upload(d, n, r)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = lfpk._stream_handle()
    v0 = views[0]
    batches = [
        [v0, synth.View(v0.pos, v0.right, v0.up, v0.fwd, v0.fov_y, 97, 61)],
        [synth.random_view(sc, 700 + k, 40 + 24 * k, 33 + 8 * k, 60.0) for k in range(6)],
    ]
    for batch in batches:
        arr, nv, total = lfpk.make_views(batch)
        want, ow = _outputs(lfp, total, dev)
        opts = lfp.lfp_render_opts()
        opts.schedule = lfp.LFP_SCHED_PERSISTENT
        opts.tile_w, opts.tile_h = 16, 8
        opts.engine = lfp.LFP_ENGINE_NESTED  # the tracer lfp_render_static runs
        lfp.lfp_render_ex(grid.handle, arr, nv, ow, opts, stream)
        got, og = _outputs(lfp, total, dev)
        st = lfp.raw_call("lfp_render_static", grid.handle, arr, nv, ctypes.byref(og), stream)
        assert st == lfp.LFP_OK, lfp.lfp_status_string(st)
        torch.cuda.synchronize()
        assert torch.equal(got["cls"], want["cls"])
        assert torch.equal(got["probe"], want["probe"])
        assert torch.equal(got["texel"], want["texel"])
        hit = (want["cls"] == 1).cpu().numpy()
        err = (got["rgb"] - want["rgb"]).abs().max(dim=1).values.cpu().numpy()
        assert hit.mean() > 0.9 and err[hit].max() <= 1e-3
        assert np.abs((got["uv"] - want["uv"]).cpu().numpy())[hit].max() <= 1e-6
    grid.close()


def test_static_render_refuses_more_views_than_its_scratch_holds():
    import paper_2507_14624_gb300 as lfpk
    from paper_2507_14624_gb300 import lfp
    sc, views, d, n, r = load_workload("tiny")
    grid = lfpk.ProbeGrid(sc.grid)
    grid.upload(d, n, r)
    many = [synth.View(views[0].pos, views[0].right, views[0].up, views[0].fwd, views[0].fov_y, 1, 1)] * (
        lfp.LFP_STATIC_MAX_VIEWS + 1)
    arr, nv, total = lfpk.make_views(many)
    dev = torch.device("cuda", torch.cuda.current_device())
    _, o = _outputs(lfp, total, dev)
    st = lfp.raw_call("lfp_render_static", grid.handle, arr, nv, ctypes.byref(o), lfpk._stream_handle())
    assert st == lfp.LFP_ERR_CAPACITY
    grid.close()
