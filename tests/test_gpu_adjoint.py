"""GPU adjoint: the scatter-add kernel against the FP64 oracle gradient and
against central finite differences of the GPU forward pass."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup(N=32, M=8, W=48, H=48):
    import paper_2507_14624_gb300 as lfpk
    g = synth.Grid(2, 2, 2, 1.0, N, M)
    sc = synth.make_scene(g, 8, 2, [1.0], seed=1)
    v = synth.random_view(sc, 101, W, H, 60.0)
    d, n, r = sc.probe_maps()
    grid = lfpk.ProbeGrid(g)
    grid.upload(d, n, r)
    return lfpk, g, sc, v, d, n, r, grid


@pytest.mark.parametrize("reduction", [1, 2, 3])
def test_adjoint_matches_fp64_oracle_gradient(reduction):
    """Per-pixel atomics, warp-aggregated atomics and the block-local sort by
    texel all give the FP64 oracle's gradient (<= 1e-4 of its largest entry)."""
    lfpk, g, sc, v, d, n, r, grid = _setup()
    views = [v, synth.random_view(sc, 77, 33, 65, 70.0)]
    out = grid.render(views)
    gr = torch.randn_like(out["rgb"])
    grad = grid.render_backward(views, gr, out["cls"], out["probe"], out["uv"], reduction=reduction)
    ref = oracle.Oracle(g, d, n, r).backward(gr.cpu().double().numpy(), out["cls"].cpu().numpy(),
                                             out["probe"].cpu().numpy(), out["uv"].cpu().double().numpy())
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(grad.cpu().numpy() - ref).max() <= 1e-4 * scale


@pytest.mark.parametrize("reduction", [1, 2, 3])
def test_adjoint_on_fp16_texels_matches_fp64_oracle_gradient(reduction):
    """FP16 radiance and normals change which texels a ray reads, not the
    adjoint: given the forward's saved state, the gradient (always FP32,
    into the caller's master copy) equals the FP64 oracle's."""
    import paper_2507_14624_gb300 as lfpk
    g = synth.Grid(2, 2, 2, 1.0, 32, 8)
    sc = synth.make_scene(g, 8, 2, [1.0], seed=1)
    d, n, r = sc.probe_maps()
    grid = lfpk.ProbeGrid(g, radiance_fmt=lfpk.LFP_TEXEL_F16, normal_fmt=lfpk.LFP_TEXEL_F16)
    grid.upload(d, n, r)
    views = [synth.random_view(sc, 101, 48, 48, 60.0), synth.random_view(sc, 77, 33, 65, 70.0)]
    out = grid.render(views)
    assert (out["cls"] == 1).float().mean().item() > 0.5
    gr = torch.randn_like(out["rgb"])
    grad = grid.render_backward(views, gr, out["cls"], out["probe"], out["uv"], reduction=reduction)
    ref = oracle.Oracle(g, d, n, r).backward(gr.cpu().double().numpy(), out["cls"].cpu().numpy(),
                                             out["probe"].cpu().numpy(), out["uv"].cpu().double().numpy())
    assert grad.dtype == torch.float32
    assert np.abs(grad.cpu().numpy() - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())


def test_adjoint_matches_central_differences_of_the_gpu_forward():
    """2x2x2 cage, 32x32 maps: rgb is linear in radiance, so the central
    difference of <g, rgb> equals the adjoint up to FP32 rounding (<= 1e-2 rel)."""
    lfpk, g, sc, v, d, n, r, grid = _setup()
    rad = torch.tensor(r, device="cuda")
    out = grid.render([v])
    gr = torch.randn_like(out["rgb"])
    grad = grid.render_backward([v], gr, out["cls"], out["probe"], out["uv"]).cpu().numpy()
    used = np.argwhere(np.abs(grad) > 1e-2)
    rng = np.random.default_rng(0)
    pick = used[rng.choice(len(used), min(30, len(used)), replace=False)]
    h = 0.25
    for p, j, i, c in pick:
        rp = rad.clone()
        rp[p, j, i, c] += h
        grid.set_radiance(rp)
        fp = (gr * grid.render([v])["rgb"]).double().sum().item()
        rm = rad.clone()
        rm[p, j, i, c] -= h
        grid.set_radiance(rm)
        fm = (gr * grid.render([v])["rgb"]).double().sum().item()
        fd = (fp - fm) / (2 * h)
        assert abs(fd - grad[p, j, i, c]) <= 1e-2 * max(abs(grad[p, j, i, c]), 1e-2)
    grid.set_radiance(rad)


def test_autograd_function_and_a_short_fit():
    """render() as a torch.autograd.Function: radiance re-initialised to
    U[0,1] is fitted back to target views by Adam on an L2 loss."""
    lfpk, g, sc, v, d, n, r, grid = _setup(N=32, M=8, W=64, H=64)
    views = [v] + [synth.random_view(sc, 900 + k, 64, 64, 60.0) for k in range(3)]
    with torch.no_grad():
        target = grid.render(views)["rgb"].clone()
    param = torch.rand((8, 32, 32, 3), device="cuda", requires_grad=True)
    opt = torch.optim.Adam([param], lr=5e-2)
    first = None
    for it in range(60):
        opt.zero_grad()
        rgb, cls = lfpk.render(param, grid, views)
        loss = ((rgb - target) ** 2).mean()
        loss.backward()
        opt.step()
        first = loss.item() if first is None else first
    assert loss.item() < 0.05 * first


def test_fit_reaches_the_noise_floor():
    """Targets = render + N(0, sigma^2); radiance re-initialised U[0,1] and
    fitted with Adam through the adjoint: the per-channel MSE on the target
    views falls to the noise floor sigma^2 (the loss is quadratic in radiance)."""
    from paper_2507_14624_gb300 import fit
    lfpk, g, sc, v, d, n, r, grid = _setup(N=32, M=8, W=64, H=64)
    views = [v] + [synth.random_view(sc, 1200 + k, 64, 64, 60.0) for k in range(7)]
    sigma = 0.01
    targets = fit.make_targets(grid, views, sigma=sigma, seed=404)
    rad, hist = fit.fit_radiance(grid, views, targets, steps=300, lr=2e-2, seed=404)
    mse = hist[-1][1]
    assert 0.5 * sigma ** 2 <= mse <= 2.0 * sigma ** 2, hist[-1]


def test_fit_checkpoint_and_resume(tmp_path):
    """A fit stopped after 6 of 12 steps and resumed from its checkpoint ends
    where the uninterrupted 12-step fit ends (up to the order of the
    adjoint's float atomics), with the history of both halves."""
    from paper_2507_14624_gb300 import fit
    lfpk, g, sc, v, d, n, r, grid = _setup(N=32, M=8, W=64, H=64)
    views = [v] + [synth.random_view(sc, 1300 + k, 48, 48, 60.0) for k in range(3)]
    targets = fit.make_targets(grid, views, sigma=0.01, seed=404)
    full, hist_full = fit.fit_radiance(grid, views, targets, steps=12, lr=2e-2, seed=7, log_every=1)
    ck = str(tmp_path / "fit.pt")
    half, _ = fit.fit_radiance(grid, views, targets, steps=6, lr=2e-2, seed=7, log_every=1, checkpoint=ck)
    assert torch.load(ck, weights_only=False)["step"] == 5
    resumed, hist = fit.fit_radiance(grid, views, targets, steps=12, lr=2e-2, seed=99, log_every=1, checkpoint=ck,
                                     checkpoint_every=4)
    assert [h[0] for h in hist] == list(range(12))
    assert torch.load(ck, weights_only=False)["step"] == 11
    assert (resumed - full).abs().max().item() <= 1e-4
    assert abs(hist[-1][1] - hist_full[-1][1]) <= 1e-6
