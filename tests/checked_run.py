"""Renders and adjoints of several configurations through the library the
binding loads (run with LFP_CHECKED=1 by test_gpu_checked.py, so through
liblfp_checked.so). Saves every output to the .npz named on the command line
and the status lfp_check_flags returned after each step."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import synth  # noqa: E402
import paper_2507_14624_gb300 as lfpk  # noqa: E402
from paper_2507_14624_gb300 import lfp  # noqa: E402


def cases():
    """(name, grid, views, render kwargs) of the checked configurations."""
    out = []
    sc, views = synth.workload("tiny")
    d, n, r = sc.probe_maps()
    g = lfpk.ProbeGrid(sc.grid)
    g.upload(d, n, r)
    mixed = views + [synth.random_view(sc, 71, 53, 29, 75.0), synth.random_view(sc, 72, 1, 7, 60.0)]
    for eng in (lfpk.LFP_ENGINE_STREAM, lfpk.LFP_ENGINE_NESTED):
        out.append((f"tiny_e{eng}", g, mixed, dict(engine=eng)))
    out.append(("tiny_flat", g, mixed, dict(engine=lfpk.LFP_ENGINE_NESTED, march=lfpk.LFP_MARCH_FLAT)))
    P = sc.grid.probe_positions()
    ge = lfpk.ProbeGrid(sc.grid, eye_lookup=lfp.LFP_EYE_NEAREST)
    ge.upload(d, n, r)
    out.append(("tiny_eye", ge, [synth.look_view(P[5], 2.1, -0.3, 70.0, 64, 48)], {}))
    sc, views = synth.workload("room")
    d, n, r = sc.probe_maps()
    for fmt in (lfpk.LFP_TEXEL_F32, lfpk.LFP_TEXEL_F16):
        gr = lfpk.ProbeGrid(sc.grid, radiance_fmt=fmt, normal_fmt=fmt)
        gr.upload(d, n, r)
        out.append((f"room_f{fmt}", gr, views, {}))
    g3 = synth.Grid(2, 2, 1, 1.0, 64, 16)
    sc3 = synth.make_scene(g3, 8, 2, [1.0], seed=21)
    d, n, r = sc3.probe_maps()
    gn = lfpk.ProbeGrid(g3, traversal=lfp.LFP_TRAVERSAL_NEAREST)
    gn.upload(d, n, r)
    out.append(("nearest", gn, [synth.random_view(sc3, 80, 96, 72, 70.0)], {}))
    return out


def main(path):
    res = {}
    for name, g, views, kw in cases():
        o = g.render(views, hit_texel=True, **kw)
        torch.cuda.synchronize()
        res[f"{name}_status"] = np.array(lfp._lib.lfp_check_flags(g.handle, None))
        for k, t in o.items():
            res[f"{name}_{k}"] = t.cpu().numpy()
        if name.startswith("tiny_e") or name == "room_f0":
            gr = torch.linspace(-1.0, 1.0, o["rgb"].numel(), device="cuda").reshape(o["rgb"].shape)
            for red in (lfp.LFP_REDUCE_ATOMIC, lfp.LFP_REDUCE_WARP, lfp.LFP_REDUCE_SORT):
                grad = g.render_backward(views, gr, o["cls"], o["probe"], o["uv"], reduction=red)
                torch.cuda.synchronize()
                res[f"{name}_bwd{red}_status"] = np.array(lfp._lib.lfp_check_flags(g.handle, None))
                res[f"{name}_bwd{red}"] = grad.cpu().numpy()
    sc, views = synth.workload("tiny")
    pc = synth.scan(sc, synth.scan_positions(sc, 2, 77), 100000, seed=9)
    gb = lfpk.ProbeGrid(sc.grid)
    gb.build_from_points(pc["xyz"], pc["rgb"], pc["normal"])
    torch.cuda.synchronize()
    res["build_status"] = np.array(lfp._lib.lfp_check_flags(gb.handle, None))
    for k, t in zip(("dist", "normal", "radiance"), gb.read_probes()):
        res[f"build_{k}"] = t.cpu().numpy()
    np.savez(path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
