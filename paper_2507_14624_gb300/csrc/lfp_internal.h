// Internal interface between the C-ABI host code and the kernel files.
#pragma once
#include <cuda_runtime.h>

#include "lfp.h"
#include "lfp_device.cuh"

namespace lfp {

constexpr int kMaxSplatProbes = 2048;
constexpr int kStreamThreadsPerBlock = 128;  // streaming engine: 4 warps per block
// Ray tiles per launch. The persistent kernels' work-queue head (an unsigned
// counter read as int) runs past the last tile by one grab per warp, plus
// the tail's half tiles: a bound far below the int range keeps it positive.
constexpr long long kMaxTilesPerLaunch = 1LL << 30;

struct RenderLaunch {
    int flat;                 // full-resolution march only (Appendix A RayMarching)
    int persistent;           // persistent CTAs pulling tiles from tile_counter
    int persistent_blocks;
    unsigned* tile_counter;   // zeroed by the caller before a persistent launch
};

cudaError_t launch_render(const GridDev& g, int rad_fmt, int nrm_fmt, const ViewBatch& vb, const OutDev& out,
                          const RenderLaunch& L, cudaStream_t s);
int render_max_active_blocks(int rad_fmt, int nrm_fmt, int threads);
// streaming engine (render_stream.cu): vb built with 8x4 ray tiles; queue
// zeroed by the caller; blocks = SMs x render_stream_blocks_per_sm; occ 0:
// 8 blocks per SM (64 registers), 1: 9 blocks per SM (56 registers)
cudaError_t launch_render_stream(const GridDev& g, int rad_fmt, int nrm_fmt, const ViewBatch& vb, const OutDev& out,
                                 unsigned* queue, int blocks, int occ, cudaStream_t s);
int render_stream_blocks_per_sm(int rad_fmt, int nrm_fmt, int occ);

// upload-time conversions: xyz normals -> octahedral RG, RGB -> RGBA texels
cudaError_t launch_encode_normals(const float* xyz, void* nrm, int nrm_fmt, long long n, cudaStream_t s);
cudaError_t launch_convert_radiance(const float* rgb, void* rad, int rad_fmt, long long n, cudaStream_t s);
// per-block min/max of the distance maps for `count` probes, into [count][2][M][M]
cudaError_t launch_build_mip(const float* dist, float* mip, int count, int N, int M, cudaStream_t s);
// least distance per quadrant of each probe's map, into qmin [count][4]
cudaError_t launch_build_qmin(const float* dist, float* qmin, int count, int N, cudaStream_t s);
// adjoint scatter into grad_radiance [P][N][N][3]; reduction: 1 per-pixel
// atomics, 2 warp-aggregated atomics, 3 block-local sort by texel. HIT
// pixels whose saved probe index is outside [0, P) are skipped and set
// kFlagBounds in *flags.
cudaError_t launch_backward(int N, int P, unsigned* flags, const PixBatch& pb, const float* grad_rgb,
                            const uint8_t* cls, const int32_t* aux_probe, const float* aux_uv, float* grad_rad,
                            int reduction, cudaStream_t s);

// probe maps from a point cloud (build_probes.cu): at most kMaxSplatProbes
// probes per splat launch (their positions sit in shared memory); keys [count][N][N] set to
// ~0 by the caller; resolve writes dist into the grid and normal xyz / rgb
// into staging planes [count][N][N][3]
cudaError_t launch_splat(const float* xyz, long long n, const GridDev& g, int first, int count,
                         unsigned long long* keys, cudaStream_t s);
cudaError_t launch_resolve(const float* xyz, const float* rgb, const float* nrm, const GridDev& g, int first,
                           int count, const unsigned long long* keys, float empty_dist, float* dist, float* nrm_out,
                           float* rgb_out, cudaStream_t s);
// read-back: stored normals -> unit xyz, stored radiance -> rgb (float32)
cudaError_t launch_decode_normals(const void* nrm, int nrm_fmt, float* xyz, long long n, cudaStream_t s);
cudaError_t launch_unpack_radiance(const void* rad, int rad_fmt, float* rgb, long long n, cudaStream_t s);

// Read-only access to a grid for render entry points outside api.cu.
struct GridAccess {
    GridDev dev;
    int rad_fmt, nrm_fmt;
    int device, sm_count;
    int all_uploaded;
};
bool grid_access(const struct lfp_grid* g, GridAccess* out);
// true if the grid keeps a skip level of block side k (lfp_skip_blocks)
bool grid_has_skip(const struct lfp_grid* g, int k);
// lfp_view -> kernel view constants (tile_w x tile_h ray tiles)
ViewDev view_dev_of(const lfp_view& v, int tile_w, int tile_h, int tile_begin);
// 0 if the views are valid (lfp_status otherwise)
int check_views_of(const lfp_view* views, int n_views);

}  // namespace lfp
