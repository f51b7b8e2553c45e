// Multi-scale hierarchy of probe grids (the multi-scale representation named
// in the abstract; the hierarchical scene representation of the teaser
// figure). Every ray of a view starts at the camera, so the level
// that traces a ray is a per-view choice: the views are grouped by level on
// the host and each group is one render (or adjoint) call on its grid, into
// the caller's shared flat outputs at each view's own out_offset.
#include <cuda_runtime.h>

#include <vector>

#include "lfp.h"
#include "lfp_internal.h"

namespace {

constexpr int kMaxLevels = 16;

// Closed box spanned by a grid's probes, in float32 as the kernels place them
// (product then sum, each rounded; volatile keeps the host compiler from
// fusing them into one multiply-add).
bool in_probe_box(const lfp::GridDev& g, const float X[3]) {
    const float o[3] = {g.ox, g.oy, g.oz};
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        volatile float ext = g.spacing * (float)(n[a] - 1);
        float hi = o[a] + ext;
        if (!(X[a] >= o[a] && X[a] <= hi)) return false;
    }
    return true;
}

// The finest level (smallest spacing, ties to the lower index) whose probe
// box holds X; if none does, the coarsest (largest spacing, ties lower).
int pick_level(const lfp::GridAccess* ga, int n_levels, const float X[3]) {
    int best = -1;
    for (int k = 0; k < n_levels; ++k)
        if (in_probe_box(ga[k].dev, X) && (best < 0 || ga[k].dev.spacing < ga[best].dev.spacing)) best = k;
    if (best >= 0) return best;
    for (int k = 0; k < n_levels; ++k)
        if (best < 0 || ga[k].dev.spacing > ga[best].dev.spacing) best = k;
    return best;
}

lfp_status gather(lfp_grid* const* levels, int n_levels, lfp::GridAccess* ga) {
    if (!levels || n_levels < 1 || n_levels > kMaxLevels) return LFP_ERR_INVALID_ARG;
    for (int k = 0; k < n_levels; ++k) {
        if (!levels[k] || !lfp::grid_access(levels[k], &ga[k])) return LFP_ERR_INVALID_ARG;
        if (ga[k].device != ga[0].device) return LFP_ERR_INVALID_ARG;
    }
    return LFP_OK;
}

// views of each level, in their input order (out_offset kept)
lfp_status group(lfp_grid* const* levels, int n_levels, const lfp_view* views, int n_views,
                 std::vector<std::vector<lfp_view>>& by_level) {
    lfp::GridAccess ga[kMaxLevels];
    lfp_status st = gather(levels, n_levels, ga);
    if (st != LFP_OK) return st;
    st = (lfp_status)lfp::check_views_of(views, n_views);
    if (st != LFP_OK) return st;
    by_level.assign(n_levels, {});
    for (int i = 0; i < n_views; ++i) by_level[pick_level(ga, n_levels, views[i].pos)].push_back(views[i]);
    return LFP_OK;
}

}  // namespace

extern "C" lfp_status lfp_pick_levels(lfp_grid* const* levels, int n_levels, const lfp_view* views, int n_views,
                                      int32_t* level_of_view) {
    if (!level_of_view) return LFP_ERR_INVALID_ARG;
    lfp::GridAccess ga[kMaxLevels];
    lfp_status st = gather(levels, n_levels, ga);
    if (st != LFP_OK) return st;
    st = (lfp_status)lfp::check_views_of(views, n_views);
    if (st != LFP_OK) return st;
    for (int i = 0; i < n_views; ++i) level_of_view[i] = pick_level(ga, n_levels, views[i].pos);
    return LFP_OK;
}

extern "C" lfp_status lfp_render_levels(lfp_grid* const* levels, int n_levels, const lfp_view* views, int n_views,
                                        const lfp_outputs* out, const lfp_render_opts* opts, void* stream) {
    if (!out) return LFP_ERR_INVALID_ARG;
    std::vector<std::vector<lfp_view>> by_level;
    lfp_status st = group(levels, n_levels, views, n_views, by_level);
    // a skip level given in opts must exist on every level that renders
    for (int k = 0; k < n_levels && st == LFP_OK; ++k)
        if (opts && opts->skip_block && !by_level[k].empty() && !lfp::grid_has_skip(levels[k], opts->skip_block))
            st = LFP_ERR_INVALID_ARG;
    for (int k = 0; k < n_levels && st == LFP_OK; ++k)
        if (!by_level[k].empty())
            st = lfp_render_ex(levels[k], by_level[k].data(), (int)by_level[k].size(), out, opts, stream);
    return st;
}

extern "C" lfp_status lfp_render_backward_levels(lfp_grid* const* levels, int n_levels, const lfp_view* views,
                                                 int n_views, const float* grad_rgb, const uint8_t* cls,
                                                 const int32_t* aux_probe, const float* aux_uv,
                                                 float* const* grad_radiance, int reduction, void* stream) {
    if (!grad_radiance) return LFP_ERR_INVALID_ARG;
    std::vector<std::vector<lfp_view>> by_level;
    lfp_status st = group(levels, n_levels, views, n_views, by_level);
    for (int k = 0; k < n_levels && st == LFP_OK; ++k)
        if (!by_level[k].empty() && !grad_radiance[k]) st = LFP_ERR_INVALID_ARG;
    for (int k = 0; k < n_levels && st == LFP_OK; ++k)
        if (!by_level[k].empty())
            st = lfp_render_backward_ex(levels[k], by_level[k].data(), (int)by_level[k].size(), grad_rgb, cls,
                                        aux_probe, aux_uv, grad_radiance[k], reduction, stream);
    return st;
}
