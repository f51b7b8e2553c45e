"""Skip levels (lfp_skip_blocks): besides the descriptor's low-resolution
map, a grid keeps min/max maps of other block sides, and the walk skips over
the blocks of one of them (Sec. 5.1's hierarchical tracing; the paper studies
the low-resolution map's size in Sec. 6). A block is skipped only while the
ray stays in front of its minimum, so every level must find the crossings the
oracle finds: each level is checked against the FP64 oracle under the
agreement rule of test_gpu_parity, the two engines against each other at
every level, and the autotuner's pick and the option checks through the
C ABI."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from conftest import load_workload
from test_gpu_parity import assert_parity, compare

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup(name):
    import paper_2507_14624_gb300 as lfpk
    sc, views, d, n, r = load_workload(name)
    trav = lfpk.lfp.LFP_TRAVERSAL_NEAREST if name == "few" else lfpk.lfp.LFP_TRAVERSAL_GRID
    grid = lfpk.ProbeGrid(sc.grid, traversal=trav)
    grid.upload(d, n, r)
    ref = oracle.Oracle(sc.grid, d, n, r, traversal=1 if name == "few" else 0).render(views[0])
    return lfpk, sc, views, grid, ref


@pytest.mark.parametrize("name", ["tiny", "room", "few"])
def test_every_skip_level_matches_oracle(name):
    lfpk, sc, views, grid, ref = _setup(name)
    ks = grid.skip_blocks
    assert sc.grid.N // sc.grid.M in ks and len(ks) >= 3, ks
    base = None
    for k in ks:
        a = grid.render(views, hit_texel=True, skip_block=k)
        st = compare(a, ref, sc.grid.N)
        print(name, "k", k, st)
        assert_parity(st)
        # the loop nest at the same level: identical decisions
        b = grid.render(views, hit_texel=True, skip_block=k, engine=lfpk.LFP_ENGINE_NESTED)
        for key in ("cls", "probe", "texel"):
            assert torch.equal(a[key], b[key]), (k, key)
        assert (a["rgb"] - b["rgb"]).abs().max().item() <= 1e-4
        # between levels only the walk's start inside a block moves: classes
        # and hit texels agree on all but near-ties
        if base is None:
            base = a
        else:
            same = (a["cls"] == base["cls"]) & (a["texel"] == base["texel"])
            assert same.float().mean().item() >= 0.9999, k


def test_skip_levels_at_non_power_of_two_block_sides():
    """k = 12 on N = 96: levels 3, 6, 12, 24 against the oracle (fuzz-style
    grid, random camera inside the cage)."""
    import paper_2507_14624_gb300 as lfpk
    g = synth.Grid(3, 2, 3, 0.5, 96, 8, (-0.3, 0.1, 0.2))
    sc = synth.make_scene(g, 24, 6, [0.7, 0.3], seed=77)
    d, n, r = sc.probe_maps()
    v = synth.random_view(sc, 177, 97, 61, 80.0)
    grid = lfpk.ProbeGrid(g)
    grid.upload(d, n, r)
    assert grid.skip_blocks == [3, 6, 12, 24]
    ref = oracle.Oracle(g, d, n, r).render(v)
    for k in grid.skip_blocks:
        st = compare(grid.render([v], hit_texel=True, skip_block=k), ref, g.N)
        assert st["disagree"] <= max(1e-3, 1.0 / v.n_pixels) and st["max_err"] <= 1e-3, (k, st)


def test_autotune_picks_a_skip_level_and_defaults_follow(room):
    import paper_2507_14624_gb300 as lfpk
    from paper_2507_14624_gb300 import lfp
    sc, views, d, n, r = room
    grid = lfpk.ProbeGrid(sc.grid)
    grid.upload(d, n, r)
    pick = grid.autotune(views)
    assert pick["skip_block"] in grid.skip_blocks, pick
    # the default now is the pick: a render with skip_block=0 equals one that names it
    a = grid.render(views, hit_texel=True)
    b = grid.render(views, hit_texel=True, skip_block=pick["skip_block"], engine=pick["engine"],
                    occupancy=pick["occupancy"], tile=pick["tile"] if pick["tile"][0] else None,
                    schedule=pick["schedule"])
    for key in ("cls", "probe", "texel", "rgb"):
        assert torch.equal(a[key], b[key]), key
    # lfp_set_defaults moves the default level; an unknown level is refused
    o = lfp.lfp_render_opts()
    o.skip_block = grid.skip_blocks[-1]
    lfp.lfp_set_defaults(grid.handle, o)
    c = grid.render(views, hit_texel=True)
    e = grid.render(views, hit_texel=True, skip_block=grid.skip_blocks[-1])
    assert torch.equal(c["texel"], e["texel"])
    o.skip_block = 5  # not a level of N = 256, M = 16
    assert lfp.raw_call("lfp_set_defaults", ctypes.c_void_p(grid.handle), ctypes.byref(o)) == lfp.LFP_ERR_INVALID_ARG
    with pytest.raises(lfp.LfpError):
        grid.render(views, skip_block=5)


def test_hierarchy_refuses_a_skip_level_missing_on_a_level():
    """lfp_render_levels checks a named skip level on every level with views
    before launching anything; a level every grid keeps renders as the
    per-grid call does."""
    import paper_2507_14624_gb300 as lfpk
    from paper_2507_14624_gb300 import lfp
    coarse = synth.Grid(2, 2, 2, 1.0, 64, 16)          # levels 2, 4, 8
    fine = synth.Grid(2, 2, 2, 0.5, 96, 8, (0.25, 0.25, 0.25))  # levels 3, 6, 12, 24
    sc = synth.make_scene(coarse, 6, 2, [1.0], seed=5)
    grids = []
    for g in (coarse, fine):
        pg = lfpk.ProbeGrid(g)
        pg.upload(*synth.level_scene(sc, g).probe_maps())
        grids.append(pg)
    views = [synth.random_view(sc, 9, 33, 17, 70.0)]
    arr, nv, total = lfpk.make_views(views)
    handles = [g.handle for g in grids]
    level = lfp.lfp_pick_levels(handles, arr, nv)[0]
    rgb = torch.empty((total, 3), dtype=torch.float32, device="cuda")
    cls = torch.empty(total, dtype=torch.uint8, device="cuda")
    o = lfp.lfp_outputs()
    o.rgb, o.cls = rgb.data_ptr(), cls.data_ptr()
    opts = lfp.lfp_render_opts()
    opts.skip_block = 5  # no grid keeps it
    with pytest.raises(lfp.LfpError) as e:
        lfp.lfp_render_levels(handles, arr, nv, o, opts, None)
    assert e.value.status == lfp.LFP_ERR_INVALID_ARG
    opts.skip_block = grids[level].skip_blocks[0]
    lfp.lfp_render_levels(handles, arr, nv, o, opts, None)
    torch.cuda.synchronize()
    want = grids[level].render(views, aux=False, skip_block=opts.skip_block)
    assert torch.equal(cls, want["cls"]) and torch.equal(rgb, want["rgb"])


@pytest.mark.parametrize("name", ["tiny", "room"])
def test_flat_march_matches_every_skip_level(name):
    """Appendix A's flat march (full-resolution map only, no skipping)
    against the hierarchical walk at every skip level, with each segment's
    walk started where the ray reaches its quadrant's least distance: the
    skips pass only texels the ray is in front of, so the decisions agree
    up to near-ties."""
    import paper_2507_14624_gb300 as lfpk
    sc, views, d, n, r = load_workload(name)
    grid = lfpk.ProbeGrid(sc.grid)
    grid.upload(d, n, r)
    flat = grid.render(views, hit_texel=True, march=lfpk.LFP_MARCH_FLAT)
    for k in grid.skip_blocks:
        for eng in (lfpk.LFP_ENGINE_STREAM, lfpk.LFP_ENGINE_NESTED):
            a = grid.render(views, hit_texel=True, skip_block=k, engine=eng)
            same = (a["cls"] == flat["cls"]) & (a["texel"] == flat["texel"])
            assert same.float().mean().item() >= 0.9999, (k, eng)


def test_hierarchy_autotune_picks_per_level():
    """ProbeHierarchy.autotune tunes each level on the views it renders; the
    picks become the levels' defaults and the images keep their decisions."""
    import paper_2507_14624_gb300 as lfpk
    coarse = synth.Grid(2, 2, 2, 1.0, 64, 16)
    fine = synth.Grid(2, 2, 2, 0.5, 96, 8, (0.25, 0.25, 0.25))
    sc = synth.make_scene(coarse, 6, 2, [1.0], seed=5)
    grids = []
    for g in (coarse, fine):
        pg = lfpk.ProbeGrid(g)
        pg.upload(*synth.level_scene(sc, g).probe_maps())
        grids.append(pg)
    h = lfpk.ProbeHierarchy(grids)
    views = [synth.random_view(sc, 90 + s, 64, 48, 70.0) for s in range(6)]
    before = h.render(views, hit_texel=True)
    picks = h.autotune(views)
    lev = h.level_of(views)
    assert set(picks) == set(lev)
    for k, p in picks.items():
        assert p["skip_block"] in grids[k].skip_blocks, (k, p)
    after = h.render(views, hit_texel=True)
    same = (before["cls"] == after["cls"]) & (before["texel"] == after["texel"])
    assert same.float().mean().item() >= 0.9999
