"""GPU parity for the paper-faithful variants against the FP64 oracle: the
traversal Sec. 4.3 gives for fewer than 8 probes, the eye-aligned texel fetch
(Appendix A traceOneProbe), and incoming-direction normal maps (Sec. 5.1).
Agreement rule as in test_gpu_parity."""
import numpy as np
import pytest

import oracle
import synth
from conftest import load_workload
from test_gpu_parity import assert_parity, compare
from test_oracle_variants import FEW_GRIDS, _cam

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _grid(sc, d, n, r, **kw):
    import paper_2507_14624_gb300 as lfpk
    g = lfpk.ProbeGrid(sc.grid, **kw)
    g.upload(d, n, r)
    return g


@pytest.mark.parametrize("dims", FEW_GRIDS)
def test_nearest_probe_traversal_matches_oracle(dims):
    """2, 4 and 8 probes, cluttered scene, several cameras plus a ragged view in
    one launch."""
    import paper_2507_14624_gb300 as lfpk
    g = synth.Grid(*dims, 1.0, 64, 16)
    sc = synth.make_scene(g, 8, 2, [1.0], seed=21)
    d, n, r = sc.probe_maps()
    views = [_cam(sc, 80 + k, 96, 72) for k in range(3)]
    views.append(synth.View(views[0].pos, views[0].right, views[0].up, views[0].fwd, views[0].fov_y, 53, 29))
    grid = _grid(sc, d, n, r, traversal=lfpk.lfp.LFP_TRAVERSAL_NEAREST)
    out = grid.render(views, hit_texel=True)
    o = oracle.Oracle(g, d, n, r, traversal=1)
    off = 0
    for v in views:
        sl = {k: t[off:off + v.n_pixels] for k, t in out.items()}
        st = compare(sl, o.render(v), g.N)
        assert st["disagree"] <= max(1e-3, 1.0 / v.n_pixels) and st["max_err"] <= 1e-3, (dims, st)
        off += v.n_pixels


def test_nearest_probe_traversal_four_probe_workload_1080p():
    import paper_2507_14624_gb300 as lfpk
    sc, views = synth.workload("few")
    d, n, r = sc.probe_maps()
    grid = _grid(sc, d, n, r, traversal=lfpk.lfp.LFP_TRAVERSAL_NEAREST)
    out = grid.render(views, hit_texel=True)
    st = compare(out, oracle.Oracle(sc.grid, d, n, r, traversal=1).render(views[0]), sc.grid.N)
    print("few", st)
    assert_parity(st)
    # the streaming engine (default) and the loop nest decide identically
    a = grid.render(views, hit_texel=True, engine=lfpk.LFP_ENGINE_NESTED)
    for k in ("cls", "probe", "texel"):
        assert torch.equal(a[k], out[k]), k
    assert (a["rgb"] - out["rgb"]).abs().max().item() <= 1e-4
    ca = grid.render(views, counters=True, engine=lfpk.LFP_ENGINE_STREAM)["counters"]
    cb = grid.render(views, counters=True, engine=lfpk.LFP_ENGINE_NESTED)["counters"]
    assert torch.equal(ca, cb)


def test_nearest_probe_traversal_refuses_more_than_eight_probes():
    import paper_2507_14624_gb300 as lfpk
    with pytest.raises(lfpk.LfpError) as e:
        lfpk.ProbeGrid(synth.Grid(3, 3, 1, 1.0, 32, 8), traversal=lfpk.lfp.LFP_TRAVERSAL_NEAREST)
    assert e.value.status == lfpk.lfp.LFP_ERR_INVALID_ARG
    with pytest.raises(lfpk.LfpError):
        lfpk.ProbeGrid(synth.Grid(2, 2, 1, 1.0, 32, 8))  # the grid iterator needs cells


@pytest.mark.parametrize("engine", [1, 2])
def test_eye_nearest_lookup_matches_oracle(tiny, engine):
    """Camera exactly at a probe with the texel fetch: every pixel takes the
    stored radiance of one texel (both engines)."""
    import paper_2507_14624_gb300 as lfpk
    sc, views, d, n, r = tiny
    P = sc.grid.probe_positions()
    v = synth.look_view(P[5], 2.1, -0.3, 70.0, 96, 80)
    grid = _grid(sc, d, n, r, eye_lookup=lfpk.lfp.LFP_EYE_NEAREST)
    out = grid.render([v], hit_texel=True, engine=engine)
    ref = oracle.Oracle(sc.grid, d, n, r, eye_nearest=True).render(v)
    assert (out["cls"].cpu().numpy() == 1).all() and (out["probe"].cpu().numpy() == 5).all()
    st = compare(out, ref, sc.grid.N)
    assert st["disagree"] <= 1e-3 and st["max_err"] <= 1e-6, st
    tex = out["texel"].cpu().numpy()
    want = r[5].reshape(-1, 3)[tex]
    agree = tex == np.where(ref["cls"] == 1, ref["texel"][:, 0] + sc.grid.N * ref["texel"][:, 1], -1)
    assert np.abs(out["rgb"].cpu().numpy()[agree] - want[agree]).max() <= 1e-6


@pytest.mark.parametrize("name", ["tiny", "room"])
def test_incoming_direction_normals_match_oracle(name):
    """Normal maps holding the incoming direction (point -> probe) instead of
    the surface normal: full frame against the oracle, streaming engine."""
    sc, views, _, _, _ = load_workload(name)
    d, n, r = sc.probe_maps(normal_mode="incoming")
    grid = _grid(sc, d, n, r)
    out = grid.render(views, hit_texel=True)
    st = compare(out, oracle.Oracle(sc.grid, d, n, r).render(views[0]), sc.grid.N)
    print(name, "incoming", st)
    assert_parity(st)


@pytest.mark.parametrize("engine", [1, 2])
def test_mixed_texel_formats(room, engine):
    """The four radiance x normal storage combinations on the room frame,
    both engines. Radiance storage never changes a decision: FP16 radiance
    with FP32 normals decides every pixel as the all-FP32 grid does, with rgb
    within FP16 rounding; FP32 radiance with FP16 normals shades every pixel
    it decides alike exactly as the all-FP32 grid does. Each combination
    meets the oracle under the FP16 rule."""
    import paper_2507_14624_gb300 as lfpk
    sc, views, d, n, r = room
    F32, F16 = lfpk.LFP_TEXEL_F32, lfpk.LFP_TEXEL_F16
    outs = {}
    for rf in (F32, F16):
        for nf in (F32, F16):
            g = _grid(sc, d, n, r, radiance_fmt=rf, normal_fmt=nf)
            outs[rf, nf] = g.render(views, hit_texel=True, engine=engine)
            g.close()
    ref = oracle.Oracle(sc.grid, d, n, r).render(views[0])
    for key, out in outs.items():
        st = compare(out, ref, sc.grid.N)
        assert st["class_match"] >= 0.999 and st["disagree"] <= 2e-3 and st["max_err"] <= 1e-3, (key, st)
    base, rad16 = outs[F32, F32], outs[F16, F32]
    for k in ("cls", "probe", "texel"):
        assert torch.equal(base[k], rad16[k]), k
    assert (base["rgb"] - rad16["rgb"]).abs().max().item() <= 1e-3
    nrm16 = outs[F32, F16]
    same = (base["cls"] == nrm16["cls"]) & (base["probe"] == nrm16["probe"]) & (base["texel"] == nrm16["texel"])
    assert same.float().mean().item() >= 0.999
    assert torch.equal(base["rgb"][same], nrm16["rgb"][same])


def test_eye_nearest_lookup_adjoint_matches_oracle(tiny):
    """The texel-fetch eye lookup samples the texel's centre, so the adjoint
    puts the whole pixel gradient on that one texel: equal to the FP64
    oracle's gradient, and every nonzero entry is a looked-up texel."""
    import paper_2507_14624_gb300 as lfpk
    sc, views, d, n, r = tiny
    P = sc.grid.probe_positions()
    v = synth.look_view(P[5], 2.1, -0.3, 70.0, 40, 30)
    grid = _grid(sc, d, n, r, eye_lookup=lfpk.lfp.LFP_EYE_NEAREST)
    out = grid.render([v], hit_texel=True)
    gr = torch.randn_like(out["rgb"])
    grad = grid.render_backward([v], gr, out["cls"], out["probe"], out["uv"])
    ref = oracle.Oracle(sc.grid, d, n, r, eye_nearest=True).backward(
        gr.cpu().double().numpy(), out["cls"].cpu().numpy(), out["probe"].cpu().numpy(),
        out["uv"].cpu().double().numpy())
    g = grad.cpu().numpy()
    assert np.abs(g - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())
    touched = np.unique(out["texel"].cpu().numpy())
    nz = np.flatnonzero(np.abs(g[5]).reshape(-1, 3).sum(1))
    assert set(nz.tolist()) <= set(touched.tolist())
    assert np.abs(np.delete(g, 5, axis=0)).max() == 0.0
