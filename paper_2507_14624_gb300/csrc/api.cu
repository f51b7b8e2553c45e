// Host side of the C ABI declared in include/lfp.h: argument checks, device
// storage owned by the grid, upload + min/max map build, batching of views
// into launches, the adjoint and the host-buffer render.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lfp.h"
#include "lfp_internal.h"

using namespace lfp;

struct lfp_grid {
    lfp_grid_desc desc;
    int P = 0;
    int device = 0;
    int sm_count = 0;
    float* dist = nullptr;
    // min/max maps per skip level (lfp_skip_blocks), block side skip_k[l],
    // each [P][2][M'][M'] with M' = N / skip_k[l]: min plane, max plane per probe
    int n_skip = 0;
    int skip_k[LFP_MAX_SKIP_LEVELS] = {};
    float* skip_mip[LFP_MAX_SKIP_LEVELS] = {};
    int skip = 0;                       // default skip level (lfp_autotune, lfp_set_defaults)
    float* qmin = nullptr;              // [P][4] least distance per map quadrant
    void* nrm = nullptr;
    void* rad = nullptr;
    unsigned* flags = nullptr;          // device flag word
    unsigned* tile_counter = nullptr;   // persistent-schedule work queue head
    float* staging = nullptr;
    size_t staging_bytes = 0;
    unsigned long long* keys = nullptr; // point-cloud builder: nearest-point table
    size_t keys_bytes = 0;
    float* cloud = nullptr;             // point-cloud builder: device copy of a host cloud
    size_t cloud_bytes = 0;
    float* host_rgb = nullptr;          // device buffers behind lfp_render_to_host
    uint8_t* host_cls = nullptr;
    long long host_pixels = 0;
    // lfp_render_to_host_async: two device output buffers used in turn, a
    // copy stream, and per buffer an event for "rendered" and "copied out"
    float* async_rgb[2] = {nullptr, nullptr};
    uint8_t* async_cls[2] = {nullptr, nullptr};
    long long async_pixels = 0;
    int async_slot = 0;
    cudaStream_t copy_stream = nullptr;
    cudaStream_t render_stream[2] = {nullptr, nullptr};  // one per buffer: consecutive frames overlap
    unsigned* async_queue = nullptr;                     // a work-queue head per render stream
    cudaEvent_t issued[2] = {nullptr, nullptr};          // the caller's stream reached the call
    cudaEvent_t rendered[2] = {nullptr, nullptr};
    cudaEvent_t copied[2] = {nullptr, nullptr};
    std::vector<unsigned char> uploaded;
    int tile_w = 16, tile_h = 8;        // default ray tile (nested engine)
    int stream_blocks[2] = {0, 0};      // persistent grid of the stream engine per register budget
    int stream_occ = 0;                 // default register budget (0: 8 blocks/SM, 1: 9; lfp_autotune)
    int engine = LFP_ENGINE_STREAM;     // default engine (set by lfp_autotune)
    int schedule = LFP_SCHED_TILES;
};

namespace {

// ---------------------------------------------------------------- helpers
std::atomic<long long> g_alloc_count{0};

// Device allocation with host-side fault injection: LFP_FAULT_ALLOC_FAIL=n
// makes the n-th allocation of the process fail with LFP_ERR_OOM before any
// CUDA call, so error paths can be tested without a GPU.
lfp_status dev_alloc(void** p, size_t bytes) {
    long long n = ++g_alloc_count;
    if (const char* f = std::getenv("LFP_FAULT_ALLOC_FAIL")) {
        long long k = std::atoll(f);
        if (k > 0 && n == k) return LFP_ERR_OOM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return LFP_ERR_OOM;
    }
    return e == cudaSuccess ? LFP_OK : LFP_ERR_CUDA;
}

void dev_free(void* p) {
    if (p) cudaFree(p);
}

#define LFP_CUDA(call)                                   \
    do {                                                 \
        if ((call) != cudaSuccess) return LFP_ERR_CUDA;  \
    } while (0)
#define LFP_TRY(call)                      \
    do {                                   \
        lfp_status st_ = (call);           \
        if (st_ != LFP_OK) return st_;     \
    } while (0)

// Makes the grid's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite3(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

size_t nrm_bytes(int fmt) { return fmt == LFP_TEXEL_F32 ? 8 : 4; }
size_t rad_bytes(int fmt) { return fmt == LFP_TEXEL_F32 ? 16 : 8; }

lfp_status check_desc(const lfp_grid_desc* d) {
    if (!d) return LFP_ERR_INVALID_ARG;
    if (d->traversal != LFP_TRAVERSAL_GRID && d->traversal != LFP_TRAVERSAL_NEAREST) return LFP_ERR_INVALID_ARG;
    if (d->eye_lookup != LFP_EYE_BILINEAR && d->eye_lookup != LFP_EYE_NEAREST) return LFP_ERR_INVALID_ARG;
    if (d->traversal == LFP_TRAVERSAL_NEAREST) {
        if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nx * d->ny * d->nz > LFP_NEAREST_MAX_PROBES)
            return LFP_ERR_INVALID_ARG;
    } else if (d->nx < 2 || d->ny < 2 || d->nz < 2 || d->nx > 4096 || d->ny > 4096 || d->nz > 4096) {
        return LFP_ERR_INVALID_ARG;
    }
    if ((long long)d->nx * d->ny * d->nz > (1LL << 24)) return LFP_ERR_INVALID_ARG;
    if (!(d->spacing > 0.0f) || !std::isfinite(d->spacing) || !finite3(d->origin)) return LFP_ERR_INVALID_ARG;
    if (d->N < 2 || d->N > 8192 || (d->N & 1)) return LFP_ERR_INVALID_ARG;
    if (d->M < 2 || d->M > d->N || (d->M & 1) || d->N % d->M) return LFP_ERR_INVALID_ARG;
    if ((d->radiance_fmt != LFP_TEXEL_F32 && d->radiance_fmt != LFP_TEXEL_F16) ||
        (d->normal_fmt != LFP_TEXEL_F32 && d->normal_fmt != LFP_TEXEL_F16))
        return LFP_ERR_INVALID_ARG;
    if (!std::isfinite(d->thickness_rel) || !std::isfinite(d->eye_eps) || d->eye_eps < 0.0f || d->max_steps < 0)
        return LFP_ERR_INVALID_ARG;
    return LFP_OK;
}

lfp_status check_views(const lfp_view* views, int n_views) {
    if (!views || n_views < 1) return LFP_ERR_INVALID_ARG;
    for (int i = 0; i < n_views; ++i) {
        const lfp_view& v = views[i];
        if (v.W < 1 || v.H < 1 || (long long)v.W * v.H > (1LL << 31) || v.out_offset < 0) return LFP_ERR_INVALID_ARG;
        if (!finite3(v.pos) || !finite3(v.right) || !finite3(v.up) || !finite3(v.fwd)) return LFP_ERR_INVALID_ARG;
        if (!(v.fov_y > 0.0f) || !(v.fov_y < 3.1415926f)) return LFP_ERR_INVALID_ARG;
    }
    return LFP_OK;
}

// Skip levels of a valid descriptor, ascending: its own block side k = N / M
// and those of k / 4, k / 2, 2 k that are whole numbers >= 2 with an even
// number of blocks per side. Returns the count; ks has room for
// LFP_MAX_SKIP_LEVELS.
int skip_levels(const lfp_grid_desc& d, int* ks) {
    const int k = d.N / d.M;
    int n = 0;
    const int cand[LFP_MAX_SKIP_LEVELS][2] = {{k, 4}, {k, 2}, {k, 1}, {2 * k, 1}};  // side = a / b
    for (auto& c : cand) {
        if (c[0] % c[1]) continue;
        const int kk = c[0] / c[1];
        if (kk != k && (kk < 2 || d.N % kk || ((d.N / kk) & 1))) continue;
        ks[n++] = kk;
    }
    return n;
}

// the skip level whose block side is k, or -1
int skip_level_of(const lfp_grid* g, int k) {
    for (int l = 0; l < g->n_skip; ++l)
        if (g->skip_k[l] == k) return l;
    return -1;
}

// level: index into g->skip_k, or -1 for the grid's default
GridDev grid_dev(const lfp_grid* g, int level = -1) {
    if (level < 0) level = g->skip;
    GridDev d;
    const lfp_grid_desc& s = g->desc;
    d.nx = s.nx;
    d.ny = s.ny;
    d.nz = s.nz;
    d.ox = s.origin[0];
    d.oy = s.origin[1];
    d.oz = s.origin[2];
    d.spacing = s.spacing;
    d.N = s.N;
    d.k = g->skip_k[level];
    d.M = s.N / d.k;
    d.kinv = (unsigned)(((1ull << 31) + (unsigned long long)d.k - 1) / (unsigned long long)d.k);
    d.two_way = s.thickness_rel < 0.0f ? 1 : 0;
    d.kappa = (float)(1.0 + 4.0 * (double)std::max(s.thickness_rel, 0.0f) / s.N);
    d.eye_eps = s.eye_eps > 0.0f ? s.eye_eps : 1e-6f * s.spacing;
    d.max_steps = s.max_steps;
    d.eye_nearest = s.eye_lookup == LFP_EYE_NEAREST ? 1 : 0;
    d.nearest_probes = s.traversal == LFP_TRAVERSAL_NEAREST ? 1 : 0;
    d.dist = g->dist;
    d.mip = g->skip_mip[level];
    d.qmin = g->qmin;
    d.nrm = g->nrm;
    d.rad = g->rad;
    d.flags = g->flags;
    return d;
}

ViewDev view_dev(const lfp_view& v, int tw, int th, int tile_begin) {
    ViewDev d;
    d.px = v.pos[0]; d.py = v.pos[1]; d.pz = v.pos[2];
    d.rx = v.right[0]; d.ry = v.right[1]; d.rz = v.right[2];
    d.ux = v.up[0]; d.uy = v.up[1]; d.uz = v.up[2];
    d.fx = v.fwd[0]; d.fy = v.fwd[1]; d.fz = v.fwd[2];
    double t = std::tan(0.5 * (double)v.fov_y);
    d.sa = (float)(t * v.W / v.H);
    d.sb = (float)t;
    d.W = v.W;
    d.H = v.H;
    d.out_offset = v.out_offset;
    d.tiles_x = (v.W + tw - 1) / tw;
    d.tile_begin = tile_begin;
    return d;
}

bool valid_tile(int w, int h) {
    return (w == 8 && h == 4) || (w == 8 && h == 8) || (w == 16 && h == 8) || (w == 16 && h == 16) ||
           (w == 32 && h == 8);
}

// queue: a work-queue head of the caller's (the frame loop's, whose launches
// overlap one another), else the grid's own.
lfp_status render_impl(lfp_grid* g, const lfp_view* views, int n_views, const OutDev& out,
                       const lfp_render_opts* opts, cudaStream_t s, unsigned* queue = nullptr) {
    // A launch alone on the GPU ends with a tail where warps run dry while
    // others still hold rays; the streaming engine hands its last tile per
    // warp out as two half tiles to even it out. Overlapping launches fill
    // each other's tails, so there the split would only add queue traffic.
    const bool overlapped = queue != nullptr;
    if (!queue) queue = g->tile_counter;  // the persistent launches' work-queue head
    int tw = g->tile_w, th = g->tile_h, sched = g->schedule, flat = 0, engine = g->engine, occ = g->stream_occ;
    int level = g->skip;
    if (opts) {
        if (opts->skip_block) {
            level = skip_level_of(g, opts->skip_block);
            if (level < 0) return LFP_ERR_INVALID_ARG;
        }
        if (opts->engine < LFP_ENGINE_AUTO || opts->engine > LFP_ENGINE_NESTED) return LFP_ERR_INVALID_ARG;
        if (opts->engine != LFP_ENGINE_AUTO) engine = opts->engine;
        if (opts->occupancy < LFP_OCC_AUTO || opts->occupancy > LFP_OCC_9) return LFP_ERR_INVALID_ARG;
        if (opts->occupancy != LFP_OCC_AUTO) occ = opts->occupancy == LFP_OCC_9 ? 1 : 0;
        if (opts->tile_w || opts->tile_h) {
            if (!valid_tile(opts->tile_w, opts->tile_h)) return LFP_ERR_INVALID_ARG;
            tw = opts->tile_w;
            th = opts->tile_h;
        }
        if (opts->march != LFP_MARCH_HIER && opts->march != LFP_MARCH_FLAT) return LFP_ERR_INVALID_ARG;
        flat = opts->march == LFP_MARCH_FLAT;
        if (opts->schedule < LFP_SCHED_AUTO || opts->schedule > LFP_SCHED_PERSISTENT) return LFP_ERR_INVALID_ARG;
        if (opts->schedule != LFP_SCHED_AUTO) sched = opts->schedule;
    }
    for (unsigned char u : g->uploaded)
        if (!u) return LFP_ERR_STATE;
    GridDev gd = grid_dev(g, level);
    static thread_local ViewBatch vb;  // ~10 KB: keep it off the host stack
    // the streaming engine runs the hierarchical march (both traversals); the
    // flat march runs on the loop nest
    if (engine == LFP_ENGINE_STREAM && !flat) {
        if (g->stream_blocks[occ] == 0)
            g->stream_blocks[occ] =
                std::max(1, render_stream_blocks_per_sm(g->desc.radiance_fmt, g->desc.normal_fmt, occ)) * g->sm_count;
        for (int first = 0; first < n_views; first += kMaxViewsPerLaunch) {
            int n = std::min(kMaxViewsPerLaunch, n_views - first);
            vb.n = n;
            vb.tile_w = 8;
            vb.tile_h = 4;
            long long tiles = 0;
            for (int i = 0; i < n; ++i) {
                const lfp_view& v = views[first + i];
                vb.v[i] = view_dev(v, 8, 4, (int)tiles);
                tiles += (long long)vb.v[i].tiles_x * ((v.H + 3) / 4);
                if (tiles > kMaxTilesPerLaunch) return LFP_ERR_INVALID_ARG;
            }
            vb.total_tiles = (int)tiles;
            int blocks = (int)std::min<long long>(g->stream_blocks[occ], (tiles + 3) / 4);
            vb.tail_tiles = overlapped ? 0 : blocks * (kStreamThreadsPerBlock / 32);
            LFP_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned), s));
            LFP_CUDA(launch_render_stream(gd, g->desc.radiance_fmt, g->desc.normal_fmt, vb, out, queue,
                                          blocks, occ, s));
        }
        return LFP_OK;
    }
    RenderLaunch L;
    L.flat = flat;
    L.persistent = sched == LFP_SCHED_PERSISTENT;
    L.tile_counter = queue;
    L.persistent_blocks = 0;
    if (L.persistent) {
        int per_sm = render_max_active_blocks(g->desc.radiance_fmt, g->desc.normal_fmt, tw * th);
        L.persistent_blocks = std::max(1, per_sm) * g->sm_count;
    }
    for (int first = 0; first < n_views; first += kMaxViewsPerLaunch) {
        int n = std::min(kMaxViewsPerLaunch, n_views - first);
        vb.n = n;
        vb.tile_w = tw;
        vb.tile_h = th;
        long long tiles = 0;
        for (int i = 0; i < n; ++i) {
            const lfp_view& v = views[first + i];
            vb.v[i] = view_dev(v, tw, th, (int)tiles);
            tiles += (long long)vb.v[i].tiles_x * ((v.H + th - 1) / th);
            if (tiles > kMaxTilesPerLaunch) return LFP_ERR_INVALID_ARG;
        }
        vb.total_tiles = (int)tiles;
        if (L.persistent) LFP_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned), s));
        LFP_CUDA(launch_render(gd, g->desc.radiance_fmt, g->desc.normal_fmt, vb, out, L, s));
    }
    return LFP_OK;
}

void destroy(lfp_grid* g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaDeviceSynchronize();
    dev_free(g->dist);
    for (float* m : g->skip_mip) dev_free(m);
    dev_free(g->qmin);
    dev_free(g->nrm);
    dev_free(g->rad);
    dev_free(g->flags);
    dev_free(g->tile_counter);
    dev_free(g->staging);
    dev_free(g->keys);
    dev_free(g->cloud);
    dev_free(g->host_rgb);
    dev_free(g->host_cls);
    for (int k = 0; k < 2; ++k) {
        dev_free(g->async_rgb[k]);
        dev_free(g->async_cls[k]);
        if (g->rendered[k]) cudaEventDestroy(g->rendered[k]);
        if (g->copied[k]) cudaEventDestroy(g->copied[k]);
        if (g->issued[k]) cudaEventDestroy(g->issued[k]);
        if (g->render_stream[k]) cudaStreamDestroy(g->render_stream[k]);
    }
    dev_free(g->async_queue);
    if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
    delete g;
}

}  // namespace

namespace lfp {

bool grid_access(const lfp_grid* g, GridAccess* out) {
    if (!g || !out) return false;
    out->dev = grid_dev(g);
    out->rad_fmt = g->desc.radiance_fmt;
    out->nrm_fmt = g->desc.normal_fmt;
    out->device = g->device;
    out->sm_count = g->sm_count;
    out->all_uploaded = 1;
    for (unsigned char u : g->uploaded)
        if (!u) out->all_uploaded = 0;
    return true;
}

bool grid_has_skip(const lfp_grid* g, int k) { return g && skip_level_of(g, k) >= 0; }

ViewDev view_dev_of(const lfp_view& v, int tile_w, int tile_h, int tile_begin) {
    return view_dev(v, tile_w, tile_h, tile_begin);
}

int check_views_of(const lfp_view* views, int n_views) { return check_views(views, n_views); }

}  // namespace lfp

namespace {

// grow a grid-owned device buffer (synchronising the stream before freeing)
template <typename T>
lfp_status ensure(T** buf, size_t* have, size_t need, cudaStream_t s) {
    if (*have >= need) return LFP_OK;
    if (*buf) {
        LFP_CUDA(cudaStreamSynchronize(s));
        dev_free(*buf);
        *buf = nullptr;
        *have = 0;
    }
    LFP_TRY(dev_alloc((void**)buf, need));
    *have = need;
    return LFP_OK;
}

// the min/max maps of probes [first, first + count) at every skip level
cudaError_t build_skip_maps(lfp_grid* g, int first, int count, cudaStream_t s) {
    const int N = g->desc.N;
    const float* dist = g->dist + (size_t)first * N * N;
    for (int l = 0; l < g->n_skip; ++l) {
        const int M = N / g->skip_k[l];
        cudaError_t e = launch_build_mip(dist, g->skip_mip[l] + (size_t)first * 2 * M * M, count, N, M, s);
        if (e != cudaSuccess) return e;
    }
    return launch_build_qmin(dist, g->qmin + (size_t)first * 4, count, N, s);
}

}  // namespace

extern "C" {

const char* lfp_status_string(lfp_status s) {
    switch (s) {
        case LFP_OK: return "ok";
        case LFP_ERR_INVALID_ARG: return "invalid argument";
        case LFP_ERR_OOM: return "out of device memory";
        case LFP_ERR_CUDA: return "CUDA error";
        case LFP_ERR_STATE: return "invalid call order (e.g. probes not uploaded)";
        case LFP_ERR_CAPACITY: return "request exceeds a fixed-size buffer (e.g. more than LFP_STATIC_MAX_VIEWS views)";
        case LFP_ERR_BOUNDS: return "an index out of range was caught (redirected to texel 0)";
        case LFP_WARN_STEPLIMIT: return "some rays reached the step limit";
    }
    return "unknown status";
}

lfp_status lfp_grid_bytes(const lfp_grid_desc* desc, unsigned long long* bytes) {
    LFP_TRY(check_desc(desc));
    if (!bytes) return LFP_ERR_INVALID_ARG;
    unsigned long long P = (unsigned long long)desc->nx * desc->ny * desc->nz;
    unsigned long long NN = (unsigned long long)desc->N * desc->N, MM = 0;
    int ks[LFP_MAX_SKIP_LEVELS];
    const int n = skip_levels(*desc, ks);
    for (int l = 0; l < n; ++l) MM += (unsigned long long)(desc->N / ks[l]) * (desc->N / ks[l]);
    *bytes = P * (NN * (4 + nrm_bytes(desc->normal_fmt) + rad_bytes(desc->radiance_fmt)) + MM * 8 + 4 * 4);
    return LFP_OK;
}

lfp_status lfp_skip_blocks(const lfp_grid_desc* desc, int* blocks, int* count) {
    LFP_TRY(check_desc(desc));
    if (!blocks || !count) return LFP_ERR_INVALID_ARG;
    *count = skip_levels(*desc, blocks);
    return LFP_OK;
}

lfp_status lfp_create_grid(const lfp_grid_desc* desc, lfp_grid** out) {
    if (!out) return LFP_ERR_INVALID_ARG;
    *out = nullptr;
    LFP_TRY(check_desc(desc));
    lfp_grid* g = new (std::nothrow) lfp_grid();
    if (!g) return LFP_ERR_OOM;
    g->desc = *desc;
    g->P = desc->nx * desc->ny * desc->nz;
    g->uploaded.assign(g->P, 0);
    size_t NN = (size_t)desc->N * desc->N;
    lfp_status st = LFP_OK;
    if (st == LFP_OK) st = dev_alloc((void**)&g->dist, g->P * NN * 4);
    g->n_skip = skip_levels(*desc, g->skip_k);
    for (int l = 0; l < g->n_skip; ++l) {
        const size_t M = desc->N / g->skip_k[l];
        if (g->skip_k[l] == desc->N / desc->M) g->skip = l;
        if (st == LFP_OK) st = dev_alloc((void**)&g->skip_mip[l], g->P * M * M * 8);
    }
    if (st == LFP_OK) st = dev_alloc((void**)&g->qmin, g->P * 4 * sizeof(float));
    if (st == LFP_OK) st = dev_alloc(&g->nrm, g->P * NN * nrm_bytes(desc->normal_fmt));
    if (st == LFP_OK) st = dev_alloc(&g->rad, g->P * NN * rad_bytes(desc->radiance_fmt));
    if (st == LFP_OK) st = dev_alloc((void**)&g->flags, 2 * sizeof(unsigned));
    if (st == LFP_OK) st = dev_alloc((void**)&g->tile_counter, sizeof(unsigned));
    if (st == LFP_OK && (cudaGetDevice(&g->device) != cudaSuccess ||
                         cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess ||
                         cudaMemset(g->flags, 0, 2 * sizeof(unsigned)) != cudaSuccess))
        st = LFP_ERR_CUDA;
    if (st != LFP_OK) {
        destroy(g);
        return st;
    }
    *out = g;
    return LFP_OK;
}

void lfp_destroy_grid(lfp_grid* g) { destroy(g); }

lfp_status lfp_upload_probes(lfp_grid* g, int first_probe, int count, const lfp_probe_planes* pl, void* stream) {
    if (!g || !pl || !pl->dist || !pl->normal || !pl->radiance) return LFP_ERR_INVALID_ARG;
    if (first_probe < 0 || count < 1 || (long long)first_probe + count > g->P) return LFP_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    if (!dg.ok) return LFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = g->desc.N;
    size_t NN = (size_t)N * N;
    float* dist_dst = g->dist + (size_t)first_probe * NN;
    char* nrm_dst = (char*)g->nrm + (size_t)first_probe * NN * nrm_bytes(g->desc.normal_fmt);
    char* rad_dst = (char*)g->rad + (size_t)first_probe * NN * rad_bytes(g->desc.radiance_fmt);
    if (pl->is_device) {
        LFP_CUDA(cudaMemcpyAsync(dist_dst, pl->dist, count * NN * 4, cudaMemcpyDeviceToDevice, s));
        LFP_CUDA(launch_encode_normals(pl->normal, nrm_dst, g->desc.normal_fmt, (long long)count * NN, s));
        LFP_CUDA(launch_convert_radiance(pl->radiance, rad_dst, g->desc.radiance_fmt, (long long)count * NN, s));
    } else {
        LFP_CUDA(cudaMemcpyAsync(dist_dst, pl->dist, count * NN * 4, cudaMemcpyHostToDevice, s));
        // xyz / rgb planes go through a grid-owned staging buffer, a few probes at a time
        size_t per_probe = NN * 3 * sizeof(float);
        int chunk = (int)std::max<size_t>(1, std::min<size_t>(count, (64u << 20) / per_probe));
        if (g->staging_bytes < chunk * per_probe) {
            LFP_CUDA(cudaStreamSynchronize(s));
            dev_free(g->staging);
            g->staging = nullptr;
            g->staging_bytes = 0;
            LFP_TRY(dev_alloc((void**)&g->staging, chunk * per_probe));
            g->staging_bytes = chunk * per_probe;
        }
        for (int c0 = 0; c0 < count; c0 += chunk) {
            int c = std::min(chunk, count - c0);
            long long n = (long long)c * NN;
            LFP_CUDA(cudaMemcpyAsync(g->staging, pl->normal + (size_t)c0 * NN * 3, n * 12, cudaMemcpyHostToDevice, s));
            LFP_CUDA(launch_encode_normals(g->staging, nrm_dst + (size_t)c0 * NN * nrm_bytes(g->desc.normal_fmt),
                                           g->desc.normal_fmt, n, s));
            LFP_CUDA(cudaMemcpyAsync(g->staging, pl->radiance + (size_t)c0 * NN * 3, n * 12, cudaMemcpyHostToDevice, s));
            LFP_CUDA(launch_convert_radiance(g->staging, rad_dst + (size_t)c0 * NN * rad_bytes(g->desc.radiance_fmt),
                                             g->desc.radiance_fmt, n, s));
        }
    }
    LFP_CUDA(build_skip_maps(g, first_probe, count, s));
    for (int p = first_probe; p < first_probe + count; ++p) g->uploaded[p] = 1;
    return LFP_OK;
}

lfp_status lfp_build_probes_from_points(lfp_grid* g, int first_probe, int count, const lfp_point_cloud* pc,
                                        float empty_dist, void* stream) {
    if (!g || !pc || !pc->xyz || !pc->rgb) return LFP_ERR_INVALID_ARG;
    if (first_probe < 0 || count < 1 || (long long)first_probe + count > g->P) return LFP_ERR_INVALID_ARG;
    if (pc->n < 1 || pc->n > 0xffffffffLL || !std::isfinite(empty_dist)) return LFP_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    if (!dg.ok) return LFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = g->desc.N;
    const size_t NN = (size_t)N * N;
    const long long n = pc->n;
    // host clouds are copied into a grid-owned device buffer (kept for the
    // next call); the copies are ordered on the stream like the kernels
    const float *xyz = pc->xyz, *rgb = pc->rgb, *nrm = pc->normal;
    if (!pc->is_device) {
        size_t planes = nrm ? 3 : 2;
        LFP_TRY(ensure(&g->cloud, &g->cloud_bytes, planes * n * 12, s));
        float* c = g->cloud;
        LFP_CUDA(cudaMemcpyAsync(c, pc->xyz, n * 12, cudaMemcpyHostToDevice, s));
        LFP_CUDA(cudaMemcpyAsync(c + 3 * n, pc->rgb, n * 12, cudaMemcpyHostToDevice, s));
        if (nrm) LFP_CUDA(cudaMemcpyAsync(c + 6 * n, pc->normal, n * 12, cudaMemcpyHostToDevice, s));
        xyz = c;
        rgb = c + 3 * n;
        nrm = nrm ? c + 6 * n : nullptr;
    }
    // chunk of probes whose key table fits a 64 MiB slice of L2
    const int chunk = (int)std::max<size_t>(
        1, std::min<size_t>(std::min(count, kMaxSplatProbes), (64u << 20) / (NN * 8)));
    lfp_status st = ensure(&g->keys, &g->keys_bytes, chunk * NN * 8, s);
    if (st == LFP_OK) st = ensure(&g->staging, &g->staging_bytes, chunk * NN * 24, s);
    GridDev gd = grid_dev(g);
    for (int c0 = 0; c0 < count && st == LFP_OK; c0 += chunk) {
        const int c = std::min(chunk, count - c0), p0 = first_probe + c0;
        const long long m = (long long)c * NN;
        float* nrm_st = g->staging;
        float* rgb_st = g->staging + 3 * m;
        cudaError_t e = cudaMemsetAsync(g->keys, 0xff, m * 8, s);
        if (e == cudaSuccess) e = launch_splat(xyz, n, gd, p0, c, g->keys, s);
        if (e == cudaSuccess)
            e = launch_resolve(xyz, rgb, nrm, gd, p0, c, g->keys, empty_dist, g->dist + (size_t)p0 * NN, nrm_st,
                               rgb_st, s);
        if (e == cudaSuccess)
            e = launch_encode_normals(nrm_st, (char*)g->nrm + (size_t)p0 * NN * nrm_bytes(g->desc.normal_fmt),
                                      g->desc.normal_fmt, m, s);
        if (e == cudaSuccess)
            e = launch_convert_radiance(rgb_st, (char*)g->rad + (size_t)p0 * NN * rad_bytes(g->desc.radiance_fmt),
                                        g->desc.radiance_fmt, m, s);
        if (e != cudaSuccess) st = LFP_ERR_CUDA;
    }
    if (st == LFP_OK && build_skip_maps(g, first_probe, count, s) != cudaSuccess) st = LFP_ERR_CUDA;
    if (st == LFP_OK)
        for (int p = first_probe; p < first_probe + count; ++p) g->uploaded[p] = 1;
    return st;
}

lfp_status lfp_read_probes(lfp_grid* g, int first_probe, int count, float* dist, float* normal, float* radiance,
                           void* stream) {
    if (!g || !dist || !normal || !radiance) return LFP_ERR_INVALID_ARG;
    if (first_probe < 0 || count < 1 || (long long)first_probe + count > g->P) return LFP_ERR_INVALID_ARG;
    for (int p = first_probe; p < first_probe + count; ++p)
        if (!g->uploaded[p]) return LFP_ERR_STATE;
    DeviceGuard dg(g->device);
    if (!dg.ok) return LFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t NN = (size_t)g->desc.N * g->desc.N;
    const long long m = (long long)count * NN;
    LFP_CUDA(cudaMemcpyAsync(dist, g->dist + (size_t)first_probe * NN, m * 4, cudaMemcpyDeviceToDevice, s));
    LFP_CUDA(launch_decode_normals((const char*)g->nrm + (size_t)first_probe * NN * nrm_bytes(g->desc.normal_fmt),
                                   g->desc.normal_fmt, normal, m, s));
    LFP_CUDA(launch_unpack_radiance((const char*)g->rad + (size_t)first_probe * NN * rad_bytes(g->desc.radiance_fmt),
                                    g->desc.radiance_fmt, radiance, m, s));
    return LFP_OK;
}

lfp_status lfp_render_ex(lfp_grid* g, const lfp_view* views, int n_views, const lfp_outputs* o,
                         const lfp_render_opts* opts, void* stream) {
    if (!g || !o) return LFP_ERR_INVALID_ARG;
    LFP_TRY(check_views(views, n_views));
    if (o->aux_uv && ((uintptr_t)o->aux_uv & 3)) return LFP_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    if (!dg.ok) return LFP_ERR_CUDA;
    OutDev out;
    out.rgb = o->rgb;
    out.cls = o->cls;
    out.aux_probe = o->aux_probe;
    out.aux_uv = o->aux_uv;
    out.hit_texel = o->hit_texel;
    out.counters = o->counters;
    return render_impl(g, views, n_views, out, opts, (cudaStream_t)stream);
}

lfp_status lfp_render(lfp_grid* g, const lfp_view* views, int n_views, float* rgb, uint8_t* cls,
                      int32_t* aux_probe, float* aux_uv, void* stream) {
    if (!rgb || !cls) return LFP_ERR_INVALID_ARG;
    lfp_outputs o;
    std::memset(&o, 0, sizeof(o));
    o.rgb = rgb;
    o.cls = cls;
    o.aux_probe = aux_probe;
    o.aux_uv = aux_uv;
    return lfp_render_ex(g, views, n_views, &o, nullptr, stream);
}

lfp_status lfp_autotune(lfp_grid* g, const lfp_view* views, int n_views, const lfp_outputs* o,
                        lfp_render_opts* best, void* stream) {
    if (!g || !o || !o->rgb || !o->cls) return LFP_ERR_INVALID_ARG;
    LFP_TRY(check_views(views, n_views));
    DeviceGuard dg(g->device);
    if (!dg.ok) return LFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    OutDev out;
    out.rgb = o->rgb;
    out.cls = o->cls;
    out.aux_probe = o->aux_probe;
    out.aux_uv = o->aux_uv;
    out.hit_texel = nullptr;
    out.counters = nullptr;
    cudaEvent_t e0, e1;
    LFP_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LFP_ERR_CUDA;
    }
    // Each candidate: one timed warm-up launch; a candidate whose warm-up
    // took more than twice the best per-launch time so far is dropped, the
    // others get one more warm-up and three timed launches.
    lfp_status st = LFP_OK;
    auto timed = [&](const lfp_render_opts& k, int reps, float* ms) -> lfp_status {
        if (cudaEventRecord(e0, s) != cudaSuccess) return LFP_ERR_CUDA;
        for (int r = 0; r < reps; ++r) LFP_TRY(render_impl(g, views, n_views, out, &k, s));
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
            return LFP_ERR_CUDA;
        return LFP_OK;
    };
    auto fastest = [&](const std::vector<lfp_render_opts>& cand, lfp_render_opts* pick) -> lfp_status {
        float best_ms = 3.4e38f;
        *pick = cand[0];
        for (const lfp_render_opts& k : cand) {
            float ms = 0.f;
            LFP_TRY(timed(k, 1, &ms));
            if (ms > 2.0f * best_ms) continue;  // clearly slower: pruned
            LFP_TRY(render_impl(g, views, n_views, out, &k, s));
            LFP_TRY(timed(k, 3, &ms));
            if (ms / 3.0f < best_ms) {
                best_ms = ms / 3.0f;
                *pick = k;
            }
        }
        return LFP_OK;
    };
    std::vector<lfp_render_opts> cand;
    lfp_render_opts c, pick;
    // 1. the skip level, on the streaming engine with the 8-block budget
    for (int l = 0; l < g->n_skip; ++l) {
        std::memset(&c, 0, sizeof(c));
        c.engine = LFP_ENGINE_STREAM;
        c.occupancy = LFP_OCC_8;
        c.skip_block = g->skip_k[l];
        cand.push_back(c);
    }
    st = fastest(cand, &pick);
    const int skip_block = pick.skip_block;
    // 2. the launch configuration at that level (the streaming candidates
    // come first and usually set the time that prunes the loop nest's)
    cand.clear();
    for (int oc : {LFP_OCC_8, LFP_OCC_9})
        if (oc == LFP_OCC_8 || g->desc.traversal == LFP_TRAVERSAL_GRID) {
            std::memset(&c, 0, sizeof(c));
            c.engine = LFP_ENGINE_STREAM;
            c.occupancy = oc;
            c.skip_block = skip_block;
            cand.push_back(c);
        }
    const int shapes[5][2] = {{8, 4}, {8, 8}, {16, 8}, {16, 16}, {32, 8}};
    for (auto& sh : shapes)
        for (int sched : {LFP_SCHED_TILES, LFP_SCHED_PERSISTENT}) {
            std::memset(&c, 0, sizeof(c));
            c.engine = LFP_ENGINE_NESTED;
            c.tile_w = sh[0];
            c.tile_h = sh[1];
            c.schedule = sched;
            c.skip_block = skip_block;
            cand.push_back(c);
        }
    if (st == LFP_OK) st = fastest(cand, &pick);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LFP_OK) return st;
    g->engine = pick.engine;
    g->skip = skip_level_of(g, pick.skip_block);
    if (pick.engine == LFP_ENGINE_STREAM) g->stream_occ = pick.occupancy == LFP_OCC_9 ? 1 : 0;
    if (pick.engine == LFP_ENGINE_NESTED) {
        g->tile_w = pick.tile_w;
        g->tile_h = pick.tile_h;
        g->schedule = pick.schedule;
    }
    if (best) *best = pick;
    return LFP_OK;
}

lfp_status lfp_set_defaults(lfp_grid* g, const lfp_render_opts* o) {
    if (!g || !o) return LFP_ERR_INVALID_ARG;
    if (o->engine < LFP_ENGINE_AUTO || o->engine > LFP_ENGINE_NESTED) return LFP_ERR_INVALID_ARG;
    if (o->occupancy < LFP_OCC_AUTO || o->occupancy > LFP_OCC_9) return LFP_ERR_INVALID_ARG;
    if (o->schedule < LFP_SCHED_AUTO || o->schedule > LFP_SCHED_PERSISTENT) return LFP_ERR_INVALID_ARG;
    if ((o->tile_w || o->tile_h) && !valid_tile(o->tile_w, o->tile_h)) return LFP_ERR_INVALID_ARG;
    if (o->march != LFP_MARCH_HIER) return LFP_ERR_INVALID_ARG;  // the flat march is a per-call diagnostic
    const int level = o->skip_block ? skip_level_of(g, o->skip_block) : g->skip;
    if (level < 0) return LFP_ERR_INVALID_ARG;
    g->skip = level;
    if (o->engine != LFP_ENGINE_AUTO) g->engine = o->engine;
    if (o->occupancy != LFP_OCC_AUTO) g->stream_occ = o->occupancy == LFP_OCC_9 ? 1 : 0;
    if (o->tile_w) {
        g->tile_w = o->tile_w;
        g->tile_h = o->tile_h;
    }
    if (o->schedule != LFP_SCHED_AUTO) g->schedule = o->schedule;
    return LFP_OK;
}

lfp_status lfp_render_to_host(lfp_grid* g, const lfp_view* views, int n_views, float* rgb_host, uint8_t* cls_host,
                              void* stream) {
    if (!g) return LFP_ERR_INVALID_ARG;
    LFP_TRY(check_views(views, n_views));
    DeviceGuard dg(g->device);
    if (!dg.ok) return LFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    long long total = 0;
    for (int i = 0; i < n_views; ++i)
        total = std::max(total, views[i].out_offset + (long long)views[i].W * views[i].H);
    if (total > g->host_pixels) {
        LFP_CUDA(cudaStreamSynchronize(s));
        dev_free(g->host_rgb);
        dev_free(g->host_cls);
        g->host_rgb = nullptr;
        g->host_cls = nullptr;
        g->host_pixels = 0;
        LFP_TRY(dev_alloc((void**)&g->host_rgb, total * 12));
        LFP_TRY(dev_alloc((void**)&g->host_cls, total));
        g->host_pixels = total;
    }
    OutDev out;
    std::memset(&out, 0, sizeof(out));
    out.rgb = g->host_rgb;
    out.cls = g->host_cls;
    LFP_TRY(render_impl(g, views, n_views, out, nullptr, s));
    if (rgb_host) LFP_CUDA(cudaMemcpyAsync(rgb_host, g->host_rgb, total * 12, cudaMemcpyDeviceToHost, s));
    if (cls_host) LFP_CUDA(cudaMemcpyAsync(cls_host, g->host_cls, total, cudaMemcpyDeviceToHost, s));
    LFP_CUDA(cudaStreamSynchronize(s));
    return LFP_OK;
}

lfp_status lfp_render_to_host_async(lfp_grid* g, const lfp_view* views, int n_views, float* rgb_host,
                                    uint8_t* cls_host, void* stream) {
    if (!g) return LFP_ERR_INVALID_ARG;
    LFP_TRY(check_views(views, n_views));
    DeviceGuard dg(g->device);
    if (!dg.ok) return LFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (!g->copy_stream) {
        LFP_TRY(dev_alloc((void**)&g->async_queue, 2 * sizeof(unsigned)));
        LFP_CUDA(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) {
            LFP_CUDA(cudaStreamCreateWithFlags(&g->render_stream[k], cudaStreamNonBlocking));
            LFP_CUDA(cudaEventCreateWithFlags(&g->issued[k], cudaEventDisableTiming));
            LFP_CUDA(cudaEventCreateWithFlags(&g->rendered[k], cudaEventDisableTiming));
            LFP_CUDA(cudaEventCreateWithFlags(&g->copied[k], cudaEventDisableTiming));
        }
    }
    long long total = 0;
    for (int i = 0; i < n_views; ++i)
        total = std::max(total, views[i].out_offset + (long long)views[i].W * views[i].H);
    if (total > g->async_pixels) {  // grow both buffers once nothing uses them
        LFP_CUDA(cudaStreamSynchronize(g->copy_stream));
        LFP_CUDA(cudaStreamSynchronize(g->render_stream[0]));
        LFP_CUDA(cudaStreamSynchronize(g->render_stream[1]));
        LFP_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < 2; ++k) {
            dev_free(g->async_rgb[k]);
            dev_free(g->async_cls[k]);
            g->async_rgb[k] = nullptr;
            g->async_cls[k] = nullptr;
        }
        g->async_pixels = 0;
        for (int k = 0; k < 2; ++k) {
            LFP_TRY(dev_alloc((void**)&g->async_rgb[k], total * 12));
            LFP_TRY(dev_alloc((void**)&g->async_cls[k], total));
        }
        g->async_pixels = total;
    }
    const int k = g->async_slot;
    g->async_slot ^= 1;
    // render k runs on its own stream after the caller's stream work so far
    // and after the buffer's previous copy (two calls ago); the other render
    // stream's frame may still be finishing, so consecutive frames overlap
    cudaStream_t rs = g->render_stream[k];
    LFP_CUDA(cudaEventRecord(g->issued[k], s));
    LFP_CUDA(cudaStreamWaitEvent(rs, g->issued[k], 0));
    LFP_CUDA(cudaStreamWaitEvent(rs, g->copied[k], 0));
    OutDev out;
    std::memset(&out, 0, sizeof(out));
    out.rgb = g->async_rgb[k];
    out.cls = g->async_cls[k];
    LFP_TRY(render_impl(g, views, n_views, out, nullptr, rs, g->async_queue + k));
    LFP_CUDA(cudaEventRecord(g->rendered[k], rs));
    LFP_CUDA(cudaStreamWaitEvent(g->copy_stream, g->rendered[k], 0));
    if (rgb_host)
        LFP_CUDA(cudaMemcpyAsync(rgb_host, g->async_rgb[k], total * 12, cudaMemcpyDeviceToHost, g->copy_stream));
    if (cls_host) LFP_CUDA(cudaMemcpyAsync(cls_host, g->async_cls[k], total, cudaMemcpyDeviceToHost, g->copy_stream));
    LFP_CUDA(cudaEventRecord(g->copied[k], g->copy_stream));
    return LFP_OK;
}

lfp_status lfp_sync_host(lfp_grid* g) {
    if (!g) return LFP_ERR_INVALID_ARG;
    if (!g->copy_stream) return LFP_OK;
    DeviceGuard dg(g->device);
    if (!dg.ok) return LFP_ERR_CUDA;
    LFP_CUDA(cudaStreamSynchronize(g->copy_stream));
    return LFP_OK;
}

lfp_status lfp_render_backward(lfp_grid* g, const lfp_view* views, int n_views, const float* grad_rgb,
                               const uint8_t* cls, const int32_t* aux_probe, const float* aux_uv,
                               float* grad_radiance, void* stream) {
    return lfp_render_backward_ex(g, views, n_views, grad_rgb, cls, aux_probe, aux_uv, grad_radiance,
                                  LFP_REDUCE_AUTO, stream);
}

lfp_status lfp_render_backward_ex(lfp_grid* g, const lfp_view* views, int n_views, const float* grad_rgb,
                                  const uint8_t* cls, const int32_t* aux_probe, const float* aux_uv,
                                  float* grad_radiance, int reduction, void* stream) {
    if (!g || !grad_rgb || !cls || !aux_probe || !aux_uv || !grad_radiance) return LFP_ERR_INVALID_ARG;
    if (reduction < LFP_REDUCE_AUTO || reduction > LFP_REDUCE_SORT) return LFP_ERR_INVALID_ARG;
    // warp aggregation: fastest measured (maps are magnified, so many pixels
    // of a warp share texels)
    if (reduction == LFP_REDUCE_AUTO) reduction = LFP_REDUCE_WARP;
    LFP_TRY(check_views(views, n_views));
    DeviceGuard dg(g->device);
    if (!dg.ok) return LFP_ERR_CUDA;
    static thread_local PixBatch pb;
    for (int first = 0; first < n_views; first += kMaxViewsPerLaunch) {
        int n = std::min(kMaxViewsPerLaunch, n_views - first);
        pb.n = n;
        pb.begin[0] = 0;
        for (int i = 0; i < n; ++i) {
            const lfp_view& v = views[first + i];
            pb.out_offset[i] = v.out_offset;
            pb.begin[i + 1] = pb.begin[i] + (long long)v.W * v.H;
        }
        LFP_CUDA(launch_backward(g->desc.N, (int)g->P, g->flags, pb, grad_rgb, cls, aux_probe, aux_uv, grad_radiance,
                                 reduction, (cudaStream_t)stream));
    }
    return LFP_OK;
}

lfp_status lfp_set_radiance(lfp_grid* g, const float* dev_rad, void* stream) {
    if (!g || !dev_rad) return LFP_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    if (!dg.ok) return LFP_ERR_CUDA;
    long long n = (long long)g->P * g->desc.N * g->desc.N;
    LFP_CUDA(launch_convert_radiance(dev_rad, g->rad, g->desc.radiance_fmt, n, (cudaStream_t)stream));
    return LFP_OK;
}

lfp_status lfp_check_flags(lfp_grid* g, void* stream) {
    if (!g) return LFP_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    if (!dg.ok) return LFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned flags = 0;
    LFP_CUDA(cudaMemcpyAsync(&flags, g->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    LFP_CUDA(cudaStreamSynchronize(s));
    LFP_CUDA(cudaMemsetAsync(g->flags, 0, sizeof(unsigned), s));
    if (flags & kFlagBounds) return LFP_ERR_BOUNDS;
    return (flags & 1u) ? LFP_WARN_STEPLIMIT : LFP_OK;
}

}  // extern "C"
