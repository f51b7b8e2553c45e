"""Batching: many views in one launch, CUDA-graph capture and the autotuner."""
import pytest

import synth
from conftest import load_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _grid(name):
    import paper_2507_14624_gb300 as lfpk
    sc, views, d, n, r = load_workload(name)
    g = lfpk.ProbeGrid(sc.grid)
    g.upload(d, n, r)
    return lfpk, sc, views, g


def _mixed_views(sc, k=7):
    sizes = [(160, 120), (64, 48), (97, 61), (200, 90), (32, 32), (150, 150), (1, 7)]
    return [synth.random_view(sc, 800 + i, *sizes[i % len(sizes)], 60.0 + 5 * i) for i in range(k)]


def test_graph_replay_equals_direct_render():
    lfpk, sc, views, g = _grid("tiny")
    vs = _mixed_views(sc)
    direct = g.render(vs, aux=True)
    graph, out = g.render_graph(vs, aux=True)
    for t in out.values():
        t.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for k in ("rgb", "cls", "probe", "uv"):
        assert torch.equal(out[k], direct[k]), k
    graph.replay()  # a second replay rewrites the same outputs
    torch.cuda.synchronize()
    assert torch.equal(out["cls"], direct["cls"])


def test_autotune_keeps_results_and_sets_a_default():
    lfpk, sc, views, g = _grid("tiny")
    vs = _mixed_views(sc, 4)
    before = g.render(vs, hit_texel=True)
    best = g.autotune(vs)
    assert best["engine"] in (lfpk.LFP_ENGINE_STREAM, lfpk.LFP_ENGINE_NESTED)
    if best["engine"] == lfpk.LFP_ENGINE_NESTED:
        assert best["tile"] in ((8, 4), (8, 8), (16, 8), (16, 16), (32, 8))
    else:
        assert best["occupancy"] in (lfpk.lfp.LFP_OCC_8, lfpk.lfp.LFP_OCC_9)
    after = g.render(vs, hit_texel=True)  # default options now follow the tuned config
    for k in ("cls", "probe", "texel"):
        assert torch.equal(before[k], after[k]), k
    assert (before["rgb"] - after["rgb"]).abs().max().item() <= 1e-4


def test_more_than_128_views_span_several_launches():
    """Views travel as kernel parameters, 128 per launch: a 300-view batch is
    split and must equal per-view renders."""
    lfpk, sc, views, g = _grid("tiny")
    vs = [synth.random_view(sc, 2000 + i, 9 + i % 5, 7 + i % 3, 60.0) for i in range(300)]
    batch = g.render(vs, hit_texel=True)
    off = 0
    for i, v in enumerate(vs):
        if i % 37 == 0:
            single = g.render([v], hit_texel=True)
            for k in ("cls", "texel"):
                assert torch.equal(batch[k][off:off + v.n_pixels], single[k]), (i, k)
        off += v.n_pixels


def test_batched_workload_full_size_sampled_against_oracle():
    """The batched configuration at full size in the launch form the bench
    times: 8x8x4 probes at N=512 with FP16 radiance and normals, 32 views of
    640x480 .. 3840x2160 (87.8 M rays), autotuned, one launch replayed from a
    CUDA graph. The replay equals a direct render; 500 sampled pixels per view
    against the FP64 oracle under the FP16 rule of test_gpu_parity
    (test_fp16_texels_error_against_fp64)."""
    import numpy as np

    import oracle
    import paper_2507_14624_gb300 as lfpk
    from test_gpu_parity import compare
    sc, views = synth.workload("batched")
    d, n, r = sc.probe_maps()
    g = lfpk.ProbeGrid(sc.grid, radiance_fmt=lfpk.LFP_TEXEL_F16, normal_fmt=lfpk.LFP_TEXEL_F16)
    g.upload(d, n, r)
    g.autotune(views)
    graph, gout = g.render_graph(views, aux=False)
    gout["cls"].fill_(255)
    graph.replay()
    direct = g.render(views, aux=True, hit_texel=True)
    torch.cuda.synchronize()
    assert torch.equal(gout["cls"], direct["cls"])
    assert torch.equal(gout["rgb"], direct["rgb"])
    o = oracle.Oracle(sc.grid, d, n, r)
    rng = np.random.default_rng(11)
    off, idx, refs = 0, [], []
    for v in views:
        pix = np.sort(rng.choice(v.n_pixels, 500, replace=False))
        refs.append(o.render(v, pix))
        idx.append(off + pix)
        off += v.n_pixels
    assert off == direct["cls"].numel()
    sel = torch.tensor(np.concatenate(idx), device="cuda")
    st = compare({k: t[sel] for k, t in direct.items()},
                 {k: np.concatenate([x[k] for x in refs]) for k in ("cls", "probe", "texel", "rgb")}, sc.grid.N)
    print("batched full size, sampled", st)
    assert st["class_match"] >= 0.999 and st["disagree"] <= 2e-3, st
    assert st["max_err"] <= 1e-3, st
    g.close()


def test_autotune_cache_applies_the_stored_pick(tmp_path):
    """A second grid of the same configuration takes the pick from the cache
    file without timing and renders exactly as the tuned grid does."""
    lfpk, sc, views, g = _grid("tiny")
    vs = _mixed_views(sc, 4)
    path = str(tmp_path / "tune.json")
    first = g.autotune(vs, cache=path)
    assert "cached" not in first
    a = g.render(vs, hit_texel=True)
    lfpk2, sc2, views2, h = _grid("tiny")
    second = h.autotune(vs, cache=path)
    assert second.get("cached") is True
    assert {k: second[k] for k in first} == first
    b = h.render(vs, hit_texel=True)
    for k in ("cls", "probe", "texel", "rgb"):
        assert torch.equal(a[k], b[k]), k
