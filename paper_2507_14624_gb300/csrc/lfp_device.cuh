// Device-side data layout and the small pieces of arithmetic shared by the
// render and adjoint kernels: octahedral encoding, texel formats, bilinear
// taps with the octahedral mirror border.
//
// Layout in HBM (one grid, P probes):
//   dist [P][N][N]  f32           radial distance (Sec. 3, r_p)
//   mip  [P][2][M][M] f32         per-block min distance (plane 0) and max
//                                 distance (plane 1): the low-resolution map
//                                 of Sec. 5.1, made conservative so skipping
//                                 is exact; the walk reads the min plane at
//                                 every low-resolution visit and the max
//                                 only at a candidate
//   qmin [P][4]     f32           per quadrant of the map, its least distance
//                                 (where a segment's low-resolution walk starts)
//   nrm  [P][N][N]  float2|half2  surface normal, octahedral-encoded
//   rad  [P][N][N]  float4|half4  radiance RGB (+ pad), 16 / 8 bytes, so the
//                                 two texels of one bilinear row are one
//                                 32-byte sector (f32) or half of one (f16)
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

namespace lfp {

enum TexFmt { kF32 = 0, kF16 = 1 };
enum Class { kMiss = 0, kHit = 1, kUnknown = 2, kStepLimit = 3 };

constexpr int kMaxViewsPerLaunch = 128;
constexpr int kNumCounters = 8;

struct GridDev {
    int nx, ny, nz;
    float ox, oy, oz, spacing;
    int N, M, k;              // k = N / M
    unsigned kinv;            // ceil(2^31 / k): exact division by k of texel indices (div_k)
    float kappa;              // crossing threshold factor 1 + 4 th / N
    int two_way;              // th < 0: every crossing goes to the normal test
    float eye_eps;
    int max_steps;            // 0 = no cap
    int eye_nearest;          // eye-aligned lookup returns the texel holding oct(w)
    int nearest_probes;       // traversal for fewer than 8 probes (Sec. 4.3)
    const float* dist;
    const float* mip;         // [P][2][M][M]
    const float* qmin;        // [P][4]: the least distance in each quadrant of the map
    const void* nrm;
    const void* rad;
    unsigned* flags;          // bit 0: step limit reached; bit 1: texel index out of range (checked builds)
};

// Checked builds (-DLFP_BOUNDS_CHECK, liblfp_checked.so) test every texel
// index of the probe maps and of the gradient before the access: an index
// out of range sets kFlagBounds in the grid's flag word and is replaced by
// texel (0, 0), so the access stays inside the map. Release builds compile
// the test away.
constexpr unsigned kFlagBounds = 2u;
#ifdef LFP_BOUNDS_CHECK
#define LFP_CHECK_TEXEL(flags, in_range, i, j)   \
    do {                                          \
        if (!(in_range)) {                        \
            atomicOr((flags), lfp::kFlagBounds);  \
            (i) = 0;                              \
            (j) = 0;                              \
        }                                         \
    } while (0)
#else
#define LFP_CHECK_TEXEL(flags, in_range, i, j) \
    do {                                        \
    } while (0)
#endif

struct ViewDev {
    float px, py, pz;
    float rx, ry, rz, ux, uy, uz, fx, fy, fz;
    float sa, sb;             // tan(fov_y / 2) * W / H, tan(fov_y / 2)
    int W, H;
    long long out_offset;
    int tiles_x;              // tiles per image row
    int tile_begin;           // first global tile index of this view
};

struct ViewBatch {
    int n;
    int total_tiles;
    int tail_tiles;  // streaming engine: the last tail_tiles tiles go out as 16-ray halves
    int tile_w, tile_h;
    ViewDev v[kMaxViewsPerLaunch];
};

// Pixel ranges of a batch of views, for per-pixel passes (the adjoint):
// batch pixel q in [begin[v], begin[v + 1]) is output index
// out_offset[v] + q - begin[v].
struct PixBatch {
    int n;
    long long begin[kMaxViewsPerLaunch + 1];
    long long out_offset[kMaxViewsPerLaunch];
};

struct OutDev {
    float* rgb;
    uint8_t* cls;
    int32_t* aux_probe;
    float* aux_uv;
    int32_t* hit_texel;
    unsigned long long* counters;
};

__device__ __forceinline__ float sgn_nz(float v) { return v >= 0.0f ? 1.0f : -1.0f; }
// Fast division and reciprocal (about 2 ulp, no special-case code path) for
// the per-ray, per-cell and per-probe set-up: short code matters more than
// the last bit there. Two places keep correctly rounded arithmetic: the
// segment set-up (its reciprocals place every texel-boundary crossing) and
// camera-ray generation. Cell faces and octant cuts use the same frcp, so a
// face through a probe is never a cut.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float frcp(float b) { return __fdividef(1.0f, b); }

// Octahedral map (Sec. 3): direction -> octahedron -> square, lower octants
// folded onto the corners (the unfold of Cigolle et al., JCGT 2014).
__device__ __forceinline__ float2 oct_encode(float x, float y, float z) {
    float l1 = fabsf(x) + fabsf(y) + fabsf(z);
    float px = fdiv(x, l1), py = fdiv(y, l1);
    if (z < 0.0f) {
        float fx = (1.0f - fabsf(py)) * sgn_nz(px);
        float fy = (1.0f - fabsf(px)) * sgn_nz(py);
        px = fx;
        py = fy;
    }
    return make_float2(px, py);
}

// Unnormalised direction of an octahedral point (enough for sign tests).
__device__ __forceinline__ float3 oct_decode_unnorm(float px, float py) {
    float z = 1.0f - fabsf(px) - fabsf(py);
    if (z < 0.0f) {
        float fx = (1.0f - fabsf(py)) * sgn_nz(px);
        float fy = (1.0f - fabsf(px)) * sgn_nz(py);
        px = fx;
        py = fy;
    }
    return make_float3(px, py, z);
}

// Octahedral mirror border: edges fold onto themselves reversed; past a
// corner, the diagonally opposite corner.
__device__ __forceinline__ void mirror_texel(int R, int& i, int& j) {
    if (i < 0) { i = 0; j = R - 1 - j; }
    else if (i >= R) { i = R - 1; j = R - 1 - j; }
    if (j < 0) { j = 0; i = R - 1 - i; }
    else if (j >= R) { j = R - 1; i = R - 1 - i; }
}

// Bilinear taps over texel centres at uv in [0,1]^2: 4 texel indices
// (i + N j) and weights, in the order (i0,j0), (i1,j0), (i0,j1), (i1,j1).
__device__ __forceinline__ void bilinear_taps(int N, float u, float v, int idx[4], float w[4]) {
    u = fminf(fmaxf(u, 0.0f), 1.0f);  // also maps NaN to 0: taps stay inside the map
    v = fminf(fmaxf(v, 0.0f), 1.0f);
    float s = u * (float)N - 0.5f, t = v * (float)N - 0.5f;
    float fs = floorf(s), ft = floorf(t);
    int i0 = (int)fs, j0 = (int)ft;
    float a = s - fs, b = t - ft;
    w[0] = (1.0f - a) * (1.0f - b);
    w[1] = a * (1.0f - b);
    w[2] = (1.0f - a) * b;
    w[3] = a * b;
    if ((unsigned)i0 < (unsigned)(N - 1) && (unsigned)j0 < (unsigned)(N - 1)) {  // all four taps inside
        const int base = i0 + N * j0;
        idx[0] = base;
        idx[1] = base + 1;
        idx[2] = base + N;
        idx[3] = base + N + 1;
        return;
    }
    int ci[4] = {i0, i0 + 1, i0, i0 + 1};
    int cj[4] = {j0, j0, j0 + 1, j0 + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int ii = ci[q], jj = cj[q];
        mirror_texel(N, ii, jj);
        idx[q] = ii + N * jj;
    }
}

template <int F> struct NrmTexel;
template <> struct NrmTexel<kF32> {
    static __device__ __forceinline__ float2 load(const void* base, size_t i) {
        return __ldg(reinterpret_cast<const float2*>(base) + i);
    }
};
template <> struct NrmTexel<kF16> {
    static __device__ __forceinline__ float2 load(const void* base, size_t i) {
        __half2 h = __ldg(reinterpret_cast<const __half2*>(base) + i);
        return __half22float2(h);
    }
};

template <int F> struct RadTexel;
template <> struct RadTexel<kF32> {
    static __device__ __forceinline__ float3 load(const void* base, size_t i) {
        float4 v = __ldg(reinterpret_cast<const float4*>(base) + i);
        return make_float3(v.x, v.y, v.z);
    }
};
template <> struct RadTexel<kF16> {
    static __device__ __forceinline__ float3 load(const void* base, size_t i) {
        uint2 raw = __ldg(reinterpret_cast<const uint2*>(base) + i);
        __half2 rg = *reinterpret_cast<__half2*>(&raw.x);
        __half2 ba = *reinterpret_cast<__half2*>(&raw.y);
        float2 a = __half22float2(rg), b = __half22float2(ba);
        return make_float3(a.x, a.y, b.x);
    }
};

// Exact x / k for 0 <= x < 8192 and 1 <= k <= 4096 by a multiply-high with
// m = ceil(2^31 / k): x m / 2^31 = x / k + x e / 2^31 with 0 <= e < 1, and
// x e / 2^31 < 1 / k whenever x k <= 2^31, so the floor is the quotient.
__device__ __forceinline__ int div_k(unsigned kinv, int x) { return (int)__umulhi((unsigned)x << 1, kinv); }

// Probe / cell-plane coordinate origin + spacing * b with two separate
// roundings (no fused multiply-add), so a cell face and a probe plane at the
// same place give bit-identical crossing times.
__device__ __forceinline__ float grid_plane(float origin, float spacing, int b) {
    return __fadd_rn(origin, __fmul_rn(spacing, (float)b));
}

}  // namespace lfp
