// Probe maps from a point cloud (Sec. 4.1 simulated probe data, Sec. 5.1
// probe data generation): every point goes into each probe's frame, is
// projected onto the octahedral map, and per texel the point nearest to the
// probe is kept. Two passes per chunk of probes:
//   splat:   one thread per point, looping over the chunk's probes; the
//            ranking key (float32 bits of |v|^2 << 32 | point index) goes to
//            the texel with a 64-bit atomicMin, skipped when the texel
//            already holds a smaller key (a stale cached read can only be
//            larger than the current minimum, so the skip is safe);
//   resolve: one thread per texel: the winner's distance, normal (its own,
//            or the incoming direction -v/|v|) and colour; empty texels get
//            empty_dist, radiance 0 and minus the texel-centre direction.
// Chunks are sized so the key table stays in L2 (64 MiB). The texel binning
// and the key are integer decisions made from floating point: they use
// explicitly rounded float32 operations (no contraction), the sequence the
// C ABI documents, so any implementation following it bins identically.
// Read-back kernels (octahedral normals -> xyz, radiance texels -> rgb)
// serve lfp_read_probes.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "lfp_internal.h"

namespace lfp {
namespace {

constexpr int kThreads = 256;

int blocks_for(long long n) { return (int)std::min<long long>((n + kThreads - 1) / kThreads, 152LL * 64); }

// Texel index of point (x, y, z) seen from probe O, or -1; q = |v|^2 and v
// on return. Every operation rounds to nearest on its own.
__device__ __forceinline__ int splat_bin(float x, float y, float z, float3 O, int N, float& q, float3& v) {
    v.x = __fsub_rn(x, O.x);
    v.y = __fsub_rn(y, O.y);
    v.z = __fsub_rn(z, O.z);
    q = __fadd_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)), __fmul_rn(v.z, v.z));
    float s = __fadd_rn(__fadd_rn(fabsf(v.x), fabsf(v.y)), fabsf(v.z));
    if (!(s > 0.0f) || !isfinite(s) || !isfinite(q)) return -1;
    const float inv = __frcp_rn(s);
    float px = __fmul_rn(v.x, inv), py = __fmul_rn(v.y, inv);
    if (v.z < 0.0f) {
        float fx = __fmul_rn(__fsub_rn(1.0f, fabsf(py)), px >= 0.0f ? 1.0f : -1.0f);
        float fy = __fmul_rn(__fsub_rn(1.0f, fabsf(px)), py >= 0.0f ? 1.0f : -1.0f);
        px = fx;
        py = fy;
    }
    const float half = (float)(N / 2);
    int i = (int)floorf(__fmul_rn(__fadd_rn(px, 1.0f), half));
    int j = (int)floorf(__fmul_rn(__fadd_rn(py, 1.0f), half));
    return min(max(i, 0), N - 1) + N * min(max(j, 0), N - 1);
}

__device__ __forceinline__ float3 probe_position(const GridDev& g, int p) {
    int ix = p % g.nx, iy = (p / g.nx) % g.ny, iz = p / (g.nx * g.ny);
    return make_float3(grid_plane(g.ox, g.spacing, ix), grid_plane(g.oy, g.spacing, iy),
                       grid_plane(g.oz, g.spacing, iz));
}

// the chunk's probe positions, once per block
__global__ void __launch_bounds__(kThreads) splat_kernel(const float* __restrict__ xyz, long long n, GridDev g,
                                                         int first, int count, unsigned long long* keys) {
    extern __shared__ float3 pos[];  // count entries
    for (int p = threadIdx.x; p < count; p += blockDim.x) pos[p] = probe_position(g, first + p);
    __syncthreads();
    const long long NN = (long long)g.N * g.N;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const float x = xyz[3 * k], y = xyz[3 * k + 1], z = xyz[3 * k + 2];
        for (int p = 0; p < count; ++p) {
            float q;
            float3 v;
            const int t = splat_bin(x, y, z, pos[p], g.N, q, v);
            if (t < 0) continue;
            const unsigned long long key = ((unsigned long long)__float_as_uint(q) << 32) | (unsigned long long)k;
            unsigned long long* slot = keys + p * NN + t;
            if (key < *slot) atomicMin(slot, key);
        }
    }
}

// dist straight into the grid; normal xyz and rgb into staging planes
__global__ void __launch_bounds__(kThreads) resolve_kernel(const float* __restrict__ xyz,
                                                           const float* __restrict__ rgb,
                                                           const float* __restrict__ nrm, GridDev g, int first,
                                                           int count, const unsigned long long* __restrict__ keys,
                                                           float empty_dist, float* dist, float* nrm_out,
                                                           float* rgb_out) {
    const long long NN = (long long)g.N * g.N, total = NN * count;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(e / NN), t = (int)(e % NN);
        const unsigned long long key = keys[e];
        float3 n;
        float3 c = make_float3(0.f, 0.f, 0.f);
        float d;
        if (key == ~0ull) {
            const int i = t % g.N, j = t / g.N;
            float3 u = oct_decode_unnorm(__fsub_rn(__fdiv_rn(2.0f * i + 1.0f, (float)g.N), 1.0f),
                                         __fsub_rn(__fdiv_rn(2.0f * j + 1.0f, (float)g.N), 1.0f));
            float l = sqrtf(u.x * u.x + u.y * u.y + u.z * u.z);
            n = make_float3(-u.x / l, -u.y / l, -u.z / l);
            d = empty_dist;
        } else {
            const long long k = (long long)(key & 0xffffffffull);
            float q;
            float3 v;
            splat_bin(xyz[3 * k], xyz[3 * k + 1], xyz[3 * k + 2], probe_position(g, first + p), g.N, q, v);
            d = __fsqrt_rn(q);
            if (nrm)
                n = make_float3(nrm[3 * k], nrm[3 * k + 1], nrm[3 * k + 2]);
            else
                n = make_float3(__fdiv_rn(-v.x, d), __fdiv_rn(-v.y, d), __fdiv_rn(-v.z, d));
            c = make_float3(rgb[3 * k], rgb[3 * k + 1], rgb[3 * k + 2]);
        }
        dist[e] = d;
        nrm_out[3 * e] = n.x;
        nrm_out[3 * e + 1] = n.y;
        nrm_out[3 * e + 2] = n.z;
        rgb_out[3 * e] = c.x;
        rgb_out[3 * e + 1] = c.y;
        rgb_out[3 * e + 2] = c.z;
    }
}

template <int F>
__global__ void decode_normals_kernel(const void* __restrict__ nrm, float* __restrict__ xyz, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 p;
        if (F == kF32) {
            p = reinterpret_cast<const float2*>(nrm)[i];
        } else {
            p = __half22float2(reinterpret_cast<const __half2*>(nrm)[i]);
        }
        float3 u = oct_decode_unnorm(p.x, p.y);
        float l = sqrtf(u.x * u.x + u.y * u.y + u.z * u.z);
        xyz[3 * i] = u.x / l;
        xyz[3 * i + 1] = u.y / l;
        xyz[3 * i + 2] = u.z / l;
    }
}

template <int F>
__global__ void unpack_radiance_kernel(const void* __restrict__ rad, float* __restrict__ rgb, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float3 c = RadTexel<F>::load(rad, (size_t)i);
        rgb[3 * i] = c.x;
        rgb[3 * i + 1] = c.y;
        rgb[3 * i + 2] = c.z;
    }
}

}  // namespace

cudaError_t launch_splat(const float* xyz, long long n, const GridDev& g, int first, int count,
                         unsigned long long* keys, cudaStream_t s) {
    if (count < 1 || count > kMaxSplatProbes) return cudaErrorInvalidValue;
    splat_kernel<<<blocks_for(n), kThreads, count * sizeof(float3), s>>>(xyz, n, g, first, count, keys);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const float* xyz, const float* rgb, const float* nrm, const GridDev& g, int first,
                           int count, const unsigned long long* keys, float empty_dist, float* dist, float* nrm_out,
                           float* rgb_out, cudaStream_t s) {
    long long total = (long long)g.N * g.N * count;
    resolve_kernel<<<blocks_for(total), kThreads, 0, s>>>(xyz, rgb, nrm, g, first, count, keys, empty_dist, dist,
                                                          nrm_out, rgb_out);
    return cudaGetLastError();
}

cudaError_t launch_decode_normals(const void* nrm, int nrm_fmt, float* xyz, long long n, cudaStream_t s) {
    if (nrm_fmt == kF32) decode_normals_kernel<kF32><<<blocks_for(n), kThreads, 0, s>>>(nrm, xyz, n);
    else decode_normals_kernel<kF16><<<blocks_for(n), kThreads, 0, s>>>(nrm, xyz, n);
    return cudaGetLastError();
}

cudaError_t launch_unpack_radiance(const void* rad, int rad_fmt, float* rgb, long long n, cudaStream_t s) {
    if (rad_fmt == kF32) unpack_radiance_kernel<kF32><<<blocks_for(n), kThreads, 0, s>>>(rad, rgb, n);
    else unpack_radiance_kernel<kF16><<<blocks_for(n), kThreads, 0, s>>>(rad, rgb, n);
    return cudaGetLastError();
}

}  // namespace lfp
