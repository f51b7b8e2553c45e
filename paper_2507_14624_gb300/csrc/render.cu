// Forward render kernel: one thread per camera ray over 2D ray tiles, one
// CTA per tile or persistent CTAs pulling tiles from a queue. The per-ray
// tracer is in render_trace.cuh.
#include <cuda_runtime.h>

#include "lfp_device.cuh"
#include "lfp_internal.h"
#include "render_trace.cuh"

namespace lfp {

namespace {

using namespace trace;

template <int RADF, int NRMF, bool COUNT, bool FLAT>
__global__ void __launch_bounds__(256) render_kernel(GridDev g, ViewBatch vb, OutDev out, int persistent,
                                                     unsigned* tile_counter) {
    __shared__ int s_tile, s_view, s_x0, s_y0;
    __shared__ ViewStart s_vs;  // the tile's view constants (all its rays start at the camera)
    const int tw = vb.tile_w, th = vb.tile_h;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wx = tw / 8;
    // warps cover 8x4 pixel sub-tiles of the ray tile
    const int lx = (warp % wx) * 8 + (lane & 7), ly = (warp / wx) * 4 + (lane >> 3);
    unsigned long long acc[kNumCounters];
    if (COUNT)
        for (int q = 0; q < kNumCounters; ++q) acc[q] = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = persistent ? (int)atomicAdd(tile_counter, 1u) : (int)blockIdx.x;
            s_tile = t;
            if (t < vb.total_tiles) {
                const int vi = view_of_tile(vb.v, vb.n, t);
                s_view = vi;
                s_vs = view_start(g, make_float3(vb.v[vi].px, vb.v[vi].py, vb.v[vi].pz), g.nearest_probes != 0);
                const int lt = t - vb.v[vi].tile_begin;  // the tile's first pixel
                s_x0 = (lt % vb.v[vi].tiles_x) * tw;
                s_y0 = (lt / vb.v[vi].tiles_x) * th;
            }
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile >= vb.total_tiles) break;
        const int lo = s_view, x0 = s_x0, y0 = s_y0;
        const ViewStart vs = s_vs;
        __syncthreads();  // s_* are rewritten by the next tile
        const ViewDev& v = vb.v[lo];
        int x = x0 + lx, y = y0 + ly;
        if (x < v.W && y < v.H) {
            float a = ((x + 0.5f) / (float)v.W * 2.0f - 1.0f) * v.sa;
            float b = (1.0f - (y + 0.5f) / (float)v.H * 2.0f) * v.sb;
            float dx = v.fx + a * v.rx + b * v.ux, dy = v.fy + a * v.ry + b * v.uy, dz = v.fz + a * v.rz + b * v.uz;
            float il = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
            Ray r;
            r.X = make_float3(v.px, v.py, v.pz);
            r.w = make_float3(dx * il, dy * il, dz * il);
            Stats<COUNT> st;
            unsigned cells = 0, probes = 0;
            PixelResult pr = trace_ray<RADF, NRMF, COUNT, FLAT>(g, r, vs, st, cells, probes);
            long long o = v.out_offset + (long long)y * v.W + x;
            if (out.rgb) {
                out.rgb[3 * o + 0] = pr.rgb.x;
                out.rgb[3 * o + 1] = pr.rgb.y;
                out.rgb[3 * o + 2] = pr.rgb.z;
            }
            if (out.cls) out.cls[o] = (uint8_t)pr.cls;
            if (out.aux_probe) out.aux_probe[o] = pr.cls == kHit ? pr.probe : -1;
            if (out.aux_uv) {
                out.aux_uv[2 * o + 0] = pr.u;
                out.aux_uv[2 * o + 1] = pr.v;
            }
            if (out.hit_texel) out.hit_texel[o] = pr.cls == kHit ? pr.texel : -1;
            if (pr.cls == kStepLimit) atomicOr(g.flags, 1u);
            if (COUNT) {
                acc[0] += st.coarse;
                acc[1] += st.fine;
                acc[2] += st.normal;
                acc[3] += pr.cls == kHit ? 4 : 0;
                acc[4] += cells;
                acc[5] += probes;
                acc[6] += pr.cls == kHit ? 1 : 0;
                acc[7] += 1;
            }
        }
        if (!persistent) break;
    }
    if (COUNT) {
        for (int q = 0; q < kNumCounters; ++q) {
            unsigned long long v = acc[q];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0 && v) atomicAdd(out.counters + q, v);
        }
    }
}

template <int RADF, int NRMF>
cudaError_t launch_fmt(const GridDev& g, const ViewBatch& vb, const OutDev& out, const RenderLaunch& L,
                       cudaStream_t s) {
    dim3 block(vb.tile_w * vb.tile_h);
    int blocks = L.persistent ? L.persistent_blocks : vb.total_tiles;
    if (blocks <= 0) return cudaSuccess;
    if (L.flat)  // diagnostic: full-resolution march only, no counters
        render_kernel<RADF, NRMF, false, true><<<blocks, block, 0, s>>>(g, vb, out, L.persistent, L.tile_counter);
    else if (out.counters)
        render_kernel<RADF, NRMF, true, false><<<blocks, block, 0, s>>>(g, vb, out, L.persistent, L.tile_counter);
    else
        render_kernel<RADF, NRMF, false, false><<<blocks, block, 0, s>>>(g, vb, out, L.persistent, L.tile_counter);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render(const GridDev& g, int rad_fmt, int nrm_fmt, const ViewBatch& vb, const OutDev& out,
                          const RenderLaunch& L, cudaStream_t s) {
    if (rad_fmt == kF32 && nrm_fmt == kF32) return launch_fmt<kF32, kF32>(g, vb, out, L, s);
    if (rad_fmt == kF16 && nrm_fmt == kF16) return launch_fmt<kF16, kF16>(g, vb, out, L, s);
    if (rad_fmt == kF16 && nrm_fmt == kF32) return launch_fmt<kF16, kF32>(g, vb, out, L, s);
    return launch_fmt<kF32, kF16>(g, vb, out, L, s);
}

int render_max_active_blocks(int rad_fmt, int nrm_fmt, int threads) {
    int n = 0;
    if (rad_fmt == kF32 && nrm_fmt == kF32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, render_kernel<kF32, kF32, false, false>, threads, 0);
    else if (rad_fmt == kF16 && nrm_fmt == kF16)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, render_kernel<kF16, kF16, false, false>, threads, 0);
    else if (rad_fmt == kF16)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, render_kernel<kF16, kF32, false, false>, threads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, render_kernel<kF32, kF16, false, false>, threads, 0);
    return n;
}

}  // namespace lfp
