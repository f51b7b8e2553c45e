// lfp_render_static: a forward render that allocates nothing.
//
// Some callers cannot allocate device memory while they render: a real-time
// frame loop that must not touch the allocator after start-up (cudaMalloc
// and cudaFree can synchronise the device and stall the loop), or a host
// application or plug-in whose device memory is handed out by its own
// fixed-budget allocator, so that a library allocating behind its back would
// break the budget. lfp_render_ex itself does not allocate, but its
// persistent schedule keeps its work-queue head in memory the grid
// allocated, and it splits large batches into several launches because
// views travel as kernel parameters. This entry point instead keeps the
// queue head and the view table in one file-scope __device__ array of fixed
// size, so one persistent launch covers up to LFP_STATIC_MAX_VIEWS views and
// the call performs no allocation of any kind. The view table is written by
// small fill kernels that carry the entries in their parameters, so the
// call reads no host memory after it returns and does not wait for the
// stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "lfp.h"
#include "lfp_device.cuh"
#include "lfp_internal.h"
#include "render_trace.cuh"

namespace lfp {
namespace {

using namespace trace;

constexpr int kTileW = 16, kTileH = 8;
constexpr size_t kHeadBytes = 256;  // queue head (word 0), rest unused
constexpr size_t kScratchBytes = kHeadBytes + (size_t)LFP_STATIC_MAX_VIEWS * sizeof(ViewDev);
// views per fill launch: 48 x 80 B of entries keep the parameter block
// under the classic 4 KB kernel-parameter limit
constexpr int kFillViews = 48;

// The scratch every call shares: queue head at offset 0, the view table at
// kHeadBytes. Each GPU that loads the library holds its own copy until the
// process exits. In host code this name is only a stand-in for the device
// address; host code uses the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_render_scratch[kScratchBytes];

// A chunk of the view table, passed by value as a kernel parameter.
struct TableChunk {
    int first, n;
    ViewDev v[kFillViews];
};
static_assert(sizeof(TableChunk) + sizeof(void*) <= 4000, "fill kernel parameters must stay under 4 KB");

__global__ void fill_table_kernel(const __grid_constant__ TableChunk c, ViewDev* table) {
    if ((int)threadIdx.x < c.n) table[c.first + threadIdx.x] = c.v[threadIdx.x];
}

template <int RADF, int NRMF, bool COUNT>
__global__ void __launch_bounds__(256) render_table_kernel(GridDev g, const ViewDev* __restrict__ views, int n_views,
                                                           int total_tiles, OutDev out, unsigned* queue) {
    __shared__ int s_tile, s_view, s_x0, s_y0;
    __shared__ ViewStart s_vs;  // the tile's view constants (all its rays start at the camera)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wx = kTileW / 8;
    const int lx = (warp % wx) * 8 + (lane & 7), ly = (warp / wx) * 4 + (lane >> 3);
    unsigned long long acc[kNumCounters];
    if (COUNT)
        for (int q = 0; q < kNumCounters; ++q) acc[q] = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = (int)atomicAdd(queue, 1u);
            s_tile = t;
            if (t < total_tiles) {
                const int vi = view_of_tile(views, n_views, t);
                s_view = vi;
                s_vs = view_start(g, make_float3(views[vi].px, views[vi].py, views[vi].pz), g.nearest_probes != 0);
                const int lt = t - views[vi].tile_begin;  // the tile's first pixel
                s_x0 = (lt % views[vi].tiles_x) * kTileW;
                s_y0 = (lt / views[vi].tiles_x) * kTileH;
            }
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile >= total_tiles) break;
        const int lo = s_view, x0 = s_x0, y0 = s_y0;
        const ViewStart vs = s_vs;
        __syncthreads();  // s_* are rewritten by the next tile
        const ViewDev v = views[lo];
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
            PixelResult pr = trace_ray<RADF, NRMF, COUNT, false>(g, r, vs, st, cells, probes);
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
    }
    if (COUNT) {
        for (int q = 0; q < kNumCounters; ++q) {
            unsigned long long v = acc[q];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0 && v) atomicAdd(out.counters + q, v);
        }
    }
}

using KernelFn = void (*)(GridDev, const ViewDev*, int, int, OutDev, unsigned*);

KernelFn pick_kernel(int rad_fmt, int nrm_fmt, bool count) {
    if (rad_fmt == kF32 && nrm_fmt == kF32)
        return count ? render_table_kernel<kF32, kF32, true> : render_table_kernel<kF32, kF32, false>;
    if (rad_fmt == kF16 && nrm_fmt == kF16)
        return count ? render_table_kernel<kF16, kF16, true> : render_table_kernel<kF16, kF16, false>;
    if (rad_fmt == kF16)
        return count ? render_table_kernel<kF16, kF32, true> : render_table_kernel<kF16, kF32, false>;
    return count ? render_table_kernel<kF32, kF16, true> : render_table_kernel<kF32, kF16, false>;
}

// Per-device set-up, done once by the first call on that device (with the
// device current): the scratch array's device address and the persistent
// grid size of each kernel variant.
constexpr int kMaxDevices = 64;
struct DeviceSetup {
    bool ready = false;
    unsigned char* scratch = nullptr;
    int blocks[2][2][2] = {};  // [rad_fmt][nrm_fmt][count]
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_mutex;  // guards g_setup; keeps one call's launches together on a stream

lfp_status setup_device(int device, int sm_count, DeviceSetup** out) {
    if (device < 0 || device >= kMaxDevices) return LFP_ERR_CUDA;
    DeviceSetup& s = g_setup[device];
    if (!s.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_render_scratch) != cudaSuccess || !p) return LFP_ERR_CUDA;
        s.scratch = static_cast<unsigned char*>(p);
        for (int rf = 0; rf < 2; ++rf)
            for (int nf = 0; nf < 2; ++nf)
                for (int c = 0; c < 2; ++c) {
                    int per_sm = 0;
                    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pick_kernel(rf, nf, c != 0),
                                                                      kTileW * kTileH, 0) != cudaSuccess)
                        return LFP_ERR_CUDA;
                    s.blocks[rf][nf][c] = std::max(1, per_sm) * sm_count;
                }
        s.ready = true;
    }
    *out = &s;
    return LFP_OK;
}

}  // namespace
}  // namespace lfp

extern "C" lfp_status lfp_render_static(lfp_grid* grid, const lfp_view* views, int n_views, const lfp_outputs* o,
                                        void* cuda_stream) {
    using namespace lfp;
    if (!grid || !o) return LFP_ERR_INVALID_ARG;
    if (n_views > LFP_STATIC_MAX_VIEWS) return LFP_ERR_CAPACITY;
    lfp_status st = (lfp_status)check_views_of(views, n_views);
    if (st != LFP_OK) return st;
    if (o->aux_uv && ((uintptr_t)o->aux_uv & 3)) return LFP_ERR_INVALID_ARG;
    GridAccess ga;
    if (!grid_access(grid, &ga)) return LFP_ERR_INVALID_ARG;
    if (!ga.all_uploaded) return LFP_ERR_STATE;
    long long tiles = 0;
    for (int i = 0; i < n_views; ++i) {
        tiles += (long long)((views[i].W + kTileW - 1) / kTileW) * ((views[i].H + kTileH - 1) / kTileH);
        if (tiles > kMaxTilesPerLaunch) return LFP_ERR_CAPACITY;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return LFP_ERR_CUDA;
    if (prev != ga.device && cudaSetDevice(ga.device) != cudaSuccess) return LFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    st = LFP_OK;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        DeviceSetup* ds = nullptr;
        st = setup_device(ga.device, ga.sm_count, &ds);
        if (st == LFP_OK) {
            unsigned* queue = reinterpret_cast<unsigned*>(ds->scratch);
            ViewDev* table = reinterpret_cast<ViewDev*>(ds->scratch + kHeadBytes);
            // the view table, kFillViews entries per fill launch (the entries
            // travel in the launch's parameters)
            TableChunk chunk;
            long long t = 0;
            for (int first = 0; first < n_views && st == LFP_OK; first += kFillViews) {
                chunk.first = first;
                chunk.n = std::min(kFillViews, n_views - first);
                for (int i = 0; i < chunk.n; ++i) {
                    const lfp_view& v = views[first + i];
                    chunk.v[i] = view_dev_of(v, kTileW, kTileH, (int)t);
                    t += (long long)chunk.v[i].tiles_x * ((v.H + kTileH - 1) / kTileH);
                }
                fill_table_kernel<<<1, kFillViews, 0, s>>>(chunk, table);
                if (cudaGetLastError() != cudaSuccess) st = LFP_ERR_CUDA;
            }
            OutDev out;
            out.rgb = o->rgb;
            out.cls = o->cls;
            out.aux_probe = o->aux_probe;
            out.aux_uv = o->aux_uv;
            out.hit_texel = o->hit_texel;
            out.counters = o->counters;
            bool count = o->counters != nullptr;
            if (st == LFP_OK && cudaMemsetAsync(queue, 0, sizeof(unsigned), s) != cudaSuccess) st = LFP_ERR_CUDA;
            if (st == LFP_OK) {
                int blocks = ds->blocks[ga.rad_fmt][ga.nrm_fmt][count ? 1 : 0];
                pick_kernel(ga.rad_fmt, ga.nrm_fmt, count)<<<blocks, kTileW * kTileH, 0, s>>>(
                    ga.dev, table, n_views, (int)tiles, out, queue);
                if (cudaGetLastError() != cudaSuccess) st = LFP_ERR_CUDA;
            }
        }
    }
    if (prev != ga.device) cudaSetDevice(prev);
    return st;
}
