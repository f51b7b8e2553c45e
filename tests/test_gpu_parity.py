"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Agreement rule: a pixel agrees when both sides give the same class and, for a
HIT, the same probe and the same full-resolution hit texel. FP32 may flip a
near-tie decision (a texel-boundary or distance tie), so at most 0.1% of
pixels may disagree; every agreeing HIT must match the oracle's radiance
within 1e-3 absolute per channel.
"""
import numpy as np
import pytest

import oracle
import synth
from conftest import load_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lfp():
    import paper_2507_14624_gb300 as lfpk
    return lfpk


def compare(out, ref, N):
    cls = out["cls"].cpu().numpy()
    probe = out["probe"].cpu().numpy()
    tex = out["texel"].cpu().numpy()
    rgb = out["rgb"].cpu().numpy().astype(np.float64)
    rtex = np.where(ref["cls"] == 1, ref["texel"][:, 0] + N * ref["texel"][:, 1], -1)
    same_cls = cls == ref["cls"]
    both_hit = (cls == 1) & (ref["cls"] == 1)
    agree_hit = both_hit & (probe == ref["probe"]) & (tex == rtex)
    disagree = ~same_cls | (both_hit & ~agree_hit)
    err = np.abs(rgb - ref["rgb"]).max(1)
    return {"class_match": same_cls.mean(), "disagree": disagree.mean(),
            "max_err": float(err[agree_hit].max()) if agree_hit.any() else 0.0,
            "hit_frac": (ref["cls"] == 1).mean(), "n": len(cls)}


def make_grid(sc, d, n, r, **kw):
    g = _lfp().ProbeGrid(sc.grid, **kw)
    g.upload(d, n, r)
    return g


def assert_parity(st, max_err=1e-3):
    assert st["class_match"] >= 0.999, st
    assert st["disagree"] <= 1e-3, st
    assert st["max_err"] <= max_err, st


def test_tiny_parity_full_frame(tiny):
    sc, views, d, n, r = tiny
    g = make_grid(sc, d, n, r)
    out = g.render(views, hit_texel=True)
    ref = oracle.Oracle(sc.grid, d, n, r).render(views[0])
    st = compare(out, ref, sc.grid.N)
    print("tiny", st)
    assert_parity(st)


def test_tiny_ragged_and_degenerate_views(tiny):
    """Views that leave partial tiles (97x61), a single pixel and a one-pixel
    wide column, rendered in one launch."""
    sc, views, d, n, r = tiny
    v0 = views[0]
    vs = [synth.View(v0.pos, v0.right, v0.up, v0.fwd, v0.fov_y, W, H) for W, H in ((97, 61), (1, 1), (1, 257))]
    g = make_grid(sc, d, n, r)
    out = g.render(vs, hit_texel=True)
    o = oracle.Oracle(sc.grid, d, n, r)
    off = 0
    for v in vs:
        ref = o.render(v)
        sl = {k: t[off:off + v.n_pixels] for k, t in out.items()}
        st = compare(sl, ref, sc.grid.N)
        assert st["disagree"] <= max(1e-3, 1.0 / v.n_pixels) and st["max_err"] <= 1e-3, (v.W, v.H, st)
        off += v.n_pixels


def test_room_parity_full_1080p(room):
    sc, views, d, n, r = room
    g = make_grid(sc, d, n, r)
    out = g.render(views, hit_texel=True)
    ref = oracle.Oracle(sc.grid, d, n, r).render(views[0])
    st = compare(out, ref, sc.grid.N)
    print("room", st)
    assert_parity(st)


@pytest.mark.parametrize("name", ["tiny", "room"])
def test_flat_march_matches_hierarchical(name):
    """Appendix A RayMarching (full-resolution only) vs low-then-full
    resolution: the min/max map only skips what the flat march passes."""
    sc, views, d, n, r = load_workload(name)
    g = make_grid(sc, d, n, r)
    lfpk = _lfp()
    a = g.render(views, hit_texel=True, march=lfpk.LFP_MARCH_HIER)
    b = g.render(views, hit_texel=True, march=lfpk.LFP_MARCH_FLAT)
    same = (a["cls"] == b["cls"]) & (a["texel"] == b["texel"])
    assert same.float().mean().item() >= 0.9999


def test_schedules_and_tile_shapes_are_identical(room):
    sc, views, d, n, r = room
    g = make_grid(sc, d, n, r)
    lfpk = _lfp()
    base = g.render(views, hit_texel=True)
    for tile in ((8, 4), (8, 8), (16, 8), (16, 16), (32, 8)):
        for sched in (lfpk.LFP_SCHED_TILES, lfpk.LFP_SCHED_PERSISTENT):
            o = g.render(views, hit_texel=True, tile=tile, schedule=sched)
            for k in ("cls", "probe", "texel", "rgb", "uv"):
                assert torch.equal(o[k], base[k]), (tile, sched, k)


@pytest.mark.parametrize("name", ["tiny", "room"])
def test_stream_engine_equals_nested_engine(name):
    """The streaming state machine and the loop nest run the same arithmetic
    on every texel: identical outputs, also for a ragged multi-view batch."""
    sc, views, d, n, r = load_workload(name)
    g = make_grid(sc, d, n, r)
    lfpk = _lfp()
    v0 = views[0]
    batch = list(views) + [synth.View(v0.pos, v0.right, v0.up, v0.fwd, v0.fov_y, 333, 121),
                           synth.random_view(sc, 4242, 250, 97, 75.0)]
    a = g.render(batch, hit_texel=True, engine=lfpk.LFP_ENGINE_STREAM)
    b = g.render(batch, hit_texel=True, engine=lfpk.LFP_ENGINE_NESTED)
    for k in ("cls", "probe", "texel"):
        assert torch.equal(a[k], b[k]), k
    # the two register budgets of the streaming engine: identical decisions;
    # the compiler may contract a multiply-add differently in each (last bit)
    c = g.render(batch, hit_texel=True, engine=lfpk.LFP_ENGINE_STREAM, occupancy=lfpk.lfp.LFP_OCC_9)
    for k in ("cls", "probe", "texel"):
        assert torch.equal(a[k], c[k]), k
    assert (a["rgb"] - c["rgb"]).abs().max().item() <= 1e-4
    assert (a["uv"] - c["uv"]).abs().max().item() <= 1e-5
    # the same formulas; multiply-add contraction may differ in the last bit
    # of the hit point, which moves the bilinear lookup by ~1e-7 texel
    assert (a["rgb"] - b["rgb"]).abs().max().item() <= 1e-4
    assert (a["uv"] - b["uv"]).abs().max().item() <= 1e-5
    ca = g.render(batch, counters=True, engine=lfpk.LFP_ENGINE_STREAM)["counters"]
    cb = g.render(batch, counters=True, engine=lfpk.LFP_ENGINE_NESTED)["counters"]
    assert torch.equal(ca, cb)


def test_batched_views_equal_single_view_launches(tiny):
    sc, views, d, n, r = tiny
    o = oracle.Oracle(sc.grid, d, n, r)
    vs = [synth.random_view(sc, 500 + k, 64 + 16 * k, 48 + 8 * k, 60.0) for k in range(5)]
    g = make_grid(sc, d, n, r)
    lfpk = _lfp()
    batch = g.render(vs, hit_texel=True, schedule=lfpk.LFP_SCHED_PERSISTENT)
    off = 0
    for v in vs:
        single = g.render([v], hit_texel=True)
        for k in ("cls", "probe", "texel", "rgb", "uv"):
            assert torch.equal(batch[k][off:off + v.n_pixels], single[k]), k
        st = compare(single, o.render(v), sc.grid.N)
        assert st["disagree"] <= 2e-3 and st["max_err"] <= 1e-3, st
        off += v.n_pixels


def test_eye_aligned_camera_on_a_probe(tiny):
    """Camera exactly at a probe: every ray is the O(1) lookup (Sec. 4.2)."""
    sc, views, d, n, r = tiny
    P = sc.grid.probe_positions()
    v = synth.look_view(P[3], 0.7, 0.2, 70.0, 96, 80)
    g = make_grid(sc, d, n, r)
    out = g.render([v], hit_texel=True)
    ref = oracle.Oracle(sc.grid, d, n, r).render(v)
    assert (out["cls"].cpu().numpy() == 1).all() and (ref["cls"] == 1).all()
    assert (out["probe"].cpu().numpy() == 3).all()
    st = compare(out, ref, sc.grid.N)
    assert st["disagree"] <= 1e-3 and st["max_err"] <= 1e-3, st


def test_device_upload_equals_host_upload(tiny):
    sc, views, d, n, r = tiny
    a = make_grid(sc, d, n, r).render(views, hit_texel=True)
    g = _lfp().ProbeGrid(sc.grid)
    g.upload(*(torch.tensor(x, device="cuda") for x in (d, n, r)))
    b = g.render(views, hit_texel=True)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_render_to_host_matches_device_render(tiny):
    sc, views, d, n, r = tiny
    g = make_grid(sc, d, n, r)
    a = g.render(views)
    P = views[0].n_pixels
    rgb = torch.empty((P, 3), dtype=torch.float32).pin_memory()
    cls = torch.empty(P, dtype=torch.uint8).pin_memory()
    g.render_to_host(views, rgb, cls)
    assert torch.equal(rgb, a["rgb"].cpu()) and torch.equal(cls, a["cls"].cpu())


def test_render_to_host_async_frame_loop(tiny):
    """Four frames (different views and sizes) through the double-buffered
    host path: after lfp_sync_host every frame's host buffers equal the
    device render of its views."""
    sc, views, d, n, r = tiny
    g = make_grid(sc, d, n, r)
    frames = [[synth.random_view(sc, 900 + k, 64 + 16 * k, 48, 60.0)] for k in range(4)]
    hosts = []
    for vs in frames:
        P = vs[0].n_pixels
        rgb = torch.empty((P, 3), dtype=torch.float32).pin_memory()
        cls = torch.empty(P, dtype=torch.uint8).pin_memory()
        g.render_to_host_async(vs, rgb, cls)
        hosts.append((rgb, cls))
    g.sync_host()
    for vs, (rgb, cls) in zip(frames, hosts):
        ref = g.render(vs)
        assert torch.equal(rgb, ref["rgb"].cpu()) and torch.equal(cls, ref["cls"].cpu())


def test_step_limit_sets_class_and_flag(tiny):
    sc, views, d, n, r = tiny
    g = make_grid(sc, d, n, r, max_steps=3)
    out = g.render(views)
    cls = out["cls"].cpu().numpy()
    assert (cls == 3).mean() > 0.5
    lfpk = _lfp()
    assert g.check_flags() == lfpk.lfp.LFP_WARN_STEPLIMIT
    assert g.check_flags() == lfpk.lfp.LFP_OK  # cleared by the read
    g2 = make_grid(sc, d, n, r)
    g2.render(views)
    assert g2.check_flags() == lfpk.lfp.LFP_OK


def test_render_before_upload_is_a_state_error(tiny):
    sc, views, d, n, r = tiny
    lfpk = _lfp()
    g = lfpk.ProbeGrid(sc.grid)
    with pytest.raises(lfpk.LfpError) as e:
        g.render(views)
    assert e.value.status == lfpk.lfp.LFP_ERR_STATE


def test_listing_two_way_rule_matches_oracle(tiny):
    """thickness_rel < 0: every crossing goes to the normal test (Appendix A
    highResolutionTracing as printed)."""
    sc, views, d, n, r = tiny
    g = make_grid(sc, d, n, r, thickness_rel=-1.0)
    out = g.render(views, hit_texel=True)
    ref = oracle.Oracle(sc.grid, d, n, r, thickness_rel=-1.0).render(views[0])
    assert_parity(compare(out, ref, sc.grid.N))


def test_fp16_texels_error_against_fp64(room):
    """FP16 radiance and normals (distance stays FP32): classification may flip
    where |n . w| is below the FP16 octahedral-normal error; radiance error is
    the FP16 rounding of values <= ~1.1 (2^-11 relative)."""
    sc, views, d, n, r = room
    lfpk = _lfp()
    g = make_grid(sc, d, n, r, radiance_fmt=lfpk.LFP_TEXEL_F16, normal_fmt=lfpk.LFP_TEXEL_F16)
    out = g.render(views, hit_texel=True)
    ref = oracle.Oracle(sc.grid, d, n, r).render(views[0])
    st = compare(out, ref, sc.grid.N)
    print("room fp16", st)
    assert st["class_match"] >= 0.999 and st["disagree"] <= 2e-3, st
    assert st["max_err"] <= 1e-3, st


def test_mixed_view_batch_in_one_launch(tiny):
    """One launch over views whose cameras sit inside the probe box, outside
    it, exactly on a probe (eye aligned) and again inside: the per-view start
    constants (eye test, first cell and its cage order) are taken once per
    tile, so tiles of different views in one launch must each get their own.
    Every view equals its own single-view launch and agrees with the oracle."""
    sc, views, d, n, r = tiny
    lfpk = _lfp()
    P = sc.grid.probe_positions()
    vs = [synth.random_view(sc, 600, 72, 40, 65.0),
          synth.look_view((-0.35, 0.41, 0.57), 0.1, 0.05, 100.0, 57, 33),
          synth.look_view(P[3], 0.7, 0.2, 70.0, 40, 24),
          synth.random_view(sc, 601, 33, 65, 80.0),
          synth.look_view((1.42, 1.37, -0.31), 3.6, 0.4, 90.0, 41, 17)]
    g = make_grid(sc, d, n, r)
    o = oracle.Oracle(sc.grid, d, n, r)
    for engine in (lfpk.LFP_ENGINE_STREAM, lfpk.LFP_ENGINE_NESTED):
        batch = g.render(vs, hit_texel=True, engine=engine, schedule=lfpk.LFP_SCHED_PERSISTENT)
        off = 0
        for v in vs:
            single = g.render([v], hit_texel=True, engine=engine)
            for k in ("cls", "probe", "texel", "rgb", "uv"):
                assert torch.equal(batch[k][off:off + v.n_pixels], single[k]), (engine, k)
            st = compare(single, o.render(v), sc.grid.N)
            assert st["disagree"] <= max(2e-3, 1.0 / v.n_pixels) and st["max_err"] <= 1e-3, (engine, st)
            off += v.n_pixels
    eye = slice(sum(v.n_pixels for v in vs[:2]), sum(v.n_pixels for v in vs[:3]))
    assert (batch["probe"][eye] == 3).all() and (batch["cls"][eye] == 1).all()
    g.close()
