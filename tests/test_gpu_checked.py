"""The checked library (liblfp_checked.so, built with -DLFP_BOUNDS_CHECK:
every texel index of a render or adjoint is tested, see lfp_check_flags) on
several configurations: no index is out of range, and the outputs equal the
release library's. Plus the adjoint's guard, in the release library, against
saved state whose probe index is outside the grid."""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_library_flags_nothing_and_matches_release(tmp_path):
    import checked_run
    import importlib.util
    spec = importlib.util.spec_from_file_location("lfp_build", os.path.join(ROOT, "paper_2507_14624_gb300", "build.py"))
    build = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(build)
    build.build(checked=True)  # up to date after __graft_entry__.build()
    chk_path, rel_path = tmp_path / "checked.npz", tmp_path / "release.npz"
    subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py"), str(chk_path)],
                   env=dict(os.environ, LFP_CHECKED="1"), cwd=ROOT, check=True, timeout=900)
    checked_run.main(str(rel_path))  # this process loaded liblfp.so
    chk, rel = np.load(chk_path), np.load(rel_path)
    assert sorted(chk.files) == sorted(rel.files)
    for k in chk.files:
        if k.endswith("_status"):
            assert int(chk[k]) == 0 and int(rel[k]) == 0, k  # LFP_OK: nothing out of range
        elif k.endswith(("_cls", "_probe", "_texel")):
            assert (chk[k] == rel[k]).mean() >= 0.9999, k  # the extra tests may change contraction
        elif k in ("build_dist", "build_radiance"):
            assert np.array_equal(chk[k], rel[k]), k
        else:
            same = np.isclose(chk[k], rel[k], rtol=1e-4, atol=1e-4)
            assert same.mean() >= 0.9999, (k, same.mean())


def test_adjoint_skips_saved_state_from_another_grid():
    """A HIT pixel whose saved probe index is past the last probe (state from
    another grid) is skipped and reported by lfp_check_flags; nothing is
    written past the gradient array."""
    import paper_2507_14624_gb300 as lfpk
    sc, views = synth.workload("tiny")
    d, n, r = sc.probe_maps()
    g = lfpk.ProbeGrid(sc.grid)
    g.upload(d, n, r)
    out = g.render(views)
    hit = torch.nonzero(out["cls"] == 1).flatten()
    assert hit.numel() > 10
    bad = hit[hit.numel() // 2].item()
    probe = out["probe"].clone()
    probe[bad] = g.n_probes
    gr = torch.randn_like(out["rgb"])
    for red in (1, 2, 3):
        room = torch.zeros((g.n_probes + 1, g.N, g.N, 3), dtype=torch.float32, device="cuda")
        g.render_backward(views, gr, out["cls"], probe, out["uv"], grad_radiance=room[:g.n_probes], reduction=red)
        with pytest.raises(lfpk.LfpError) as e:
            g.check_flags()
        assert e.value.status == lfpk.lfp.LFP_ERR_BOUNDS
        assert g.check_flags() == lfpk.lfp.LFP_OK  # the flag word was cleared
        assert room[g.n_probes].abs().max().item() == 0.0
        cls = out["cls"].clone()
        cls[bad] = 0  # the same pixels without the bad one
        ref = g.render_backward(views, gr, cls, out["probe"], out["uv"], reduction=red)
        assert torch.allclose(room[:g.n_probes], ref, rtol=1e-5, atol=1e-5)
    g.close()
