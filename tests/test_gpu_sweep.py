"""GPU parity at the map sizes of the resolution study (Sec. 6: full-
resolution maps N in {1024, 2048, 3072}, low-resolution maps M in {64, 128}):
the room grid (4x4x4 probes at spacing 0.5, the room scene, ray-cast maps)
rendered through the C ABI with the grid traversal and compared with the
FP64 oracle on every pixel of the room view at 320x180, under the agreement
rule of test_gpu_parity. The block sides k = N / M are 16, 8, 32, 16 and the
non-powers of two 48 and 24."""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import assert_parity, compare

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("N", [1024, 2048, 3072])
def test_sweep_map_sizes_match_oracle(N):
    import paper_2507_14624_gb300 as lfpk
    sc, views = synth.workload("room")
    v0 = views[0]
    v = synth.View(v0.pos, v0.right, v0.up, v0.fwd, v0.fov_y, 320, 180)
    d, n, r = sc.probe_maps(N=N)  # every probe of the room grid at this map side
    for M in (64, 128):
        g = synth.Grid(4, 4, 4, 0.5, N, M)
        grid = lfpk.ProbeGrid(g)
        grid.upload(d, n, r)
        out = grid.render([v], hit_texel=True)
        ref = oracle.Oracle(g, d, n, r).render(v)
        st = compare(out, ref, N)
        print(f"N={N} M={M} k={N // M}", st)
        assert_parity(st)
        grid.close()
        del grid, out
        torch.cuda.empty_cache()
