// Upload-time conversions, the min/max low-resolution map and the adjoint.
#include <cuda_runtime.h>

#include <algorithm>

#include "lfp_device.cuh"
#include "lfp_internal.h"

namespace lfp {

namespace {

constexpr int kThreads = 256;

int blocks_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > (1LL << 30) ? (1LL << 30) : b));
}

template <int F>
__global__ void encode_normals_kernel(const float* __restrict__ xyz, void* __restrict__ nrm, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 p = oct_encode(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
        if (F == kF32)
            reinterpret_cast<float2*>(nrm)[i] = p;
        else
            reinterpret_cast<__half2*>(nrm)[i] = __floats2half2_rn(p.x, p.y);
    }
}

template <int F>
__global__ void convert_radiance_kernel(const float* __restrict__ rgb, void* __restrict__ rad, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float r = rgb[3 * i], g = rgb[3 * i + 1], b = rgb[3 * i + 2];
        if (F == kF32) {
            reinterpret_cast<float4*>(rad)[i] = make_float4(r, g, b, 0.0f);
        } else {
            __half2 rg = __floats2half2_rn(r, g), ba = __floats2half2_rn(b, 0.0f);
            uint2 raw;
            raw.x = *reinterpret_cast<unsigned*>(&rg);
            raw.y = *reinterpret_cast<unsigned*>(&ba);
            reinterpret_cast<uint2*>(rad)[i] = raw;
        }
    }
}

// one thread per coarse texel: min and max over its k x k block
__global__ void build_mip_kernel(const float* __restrict__ dist, float* __restrict__ mip, int count, int N, int M) {
    long long total = (long long)count * M * M;
    int k = N / M;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total; c += (long long)gridDim.x * blockDim.x) {
        int p = (int)(c / ((long long)M * M));
        int rem = (int)(c % ((long long)M * M));
        int J = rem / M, I = rem % M;
        const float* base = dist + (size_t)p * N * N;
        float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
        for (int j = J * k; j < (J + 1) * k; ++j)
            for (int i = I * k; i < (I + 1) * k; ++i) {
                float v = base[(size_t)j * N + i];
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
            }
        float* page = mip + (size_t)p * 2 * M * M;  // this probe's min plane, then its max plane
        page[rem] = lo;
        page[(size_t)M * M + rem] = hi;
    }
}

// Least distance of each quadrant of each probe's map: one block per
// (probe, quadrant).
__global__ void build_qmin_kernel(const float* __restrict__ dist, float* __restrict__ qmin, int N) {
    const int p = blockIdx.x >> 2, q = blockIdx.x & 3, h = N / 2;
    const float* base = dist + (size_t)p * N * N + (size_t)((q & 2) ? h : 0) * N + ((q & 1) ? h : 0);
    float lo = __int_as_float(0x7f800000);
    for (int t = threadIdx.x; t < h * h; t += blockDim.x) lo = fminf(lo, base[(size_t)(t / h) * N + t % h]);
    for (int off = 16; off > 0; off >>= 1) lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    __shared__ float part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) lo = fminf(lo, part[w]);
        qmin[blockIdx.x] = fminf(lo, part[0]);
    }
}

// Adjoint: for every HIT pixel add w_k * g_c into the 4 bilinear taps.
__global__ void backward_kernel(int N, int P, unsigned* flags, PixBatch pb, const float* __restrict__ grad_rgb,
                                const uint8_t* __restrict__ cls, const int32_t* __restrict__ aux_probe,
                                const float* __restrict__ aux_uv, float* __restrict__ grad_rad) {
    long long total = pb.begin[pb.n];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = pb.n - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (pb.begin[mid] <= q) lo = mid; else hi = mid - 1;
        }
        long long o = pb.out_offset[lo] + (q - pb.begin[lo]);
        if (cls[o] != kHit) continue;
        int p = aux_probe[o];
        if ((unsigned)p >= (unsigned)P) {  // not the saved state of a render of this grid
            atomicOr(flags, kFlagBounds);
            continue;
        }
        int idx[4];
        float w[4];
        bilinear_taps(N, aux_uv[2 * o], aux_uv[2 * o + 1], idx, w);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int zero = 0;
            LFP_CHECK_TEXEL(flags, (unsigned)idx[k] < (unsigned)(N * N), idx[k], zero);
        }
        float g0 = grad_rgb[3 * o], g1 = grad_rgb[3 * o + 1], g2 = grad_rgb[3 * o + 2];
        float* base = grad_rad + (size_t)p * N * N * 3;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float* t = base + 3 * (size_t)idx[k];
            atomicAdd(t + 0, w[k] * g0);
            atomicAdd(t + 1, w[k] * g1);
            atomicAdd(t + 2, w[k] * g2);
        }
    }
}

// Warp-aggregated adjoint: pixels of one warp that hit the same texel (the
// maps are magnified: hundreds of pixels per texel at 1080p) are summed and
// written by one atomic per texel and channel. A warp holds 32 consecutive
// pixels of a row, so equal texels come in runs of neighbouring lanes: a
// segmented sum over the runs (five shuffle steps) leaves each run's total
// in its last lane, which does the atomics.
__global__ void backward_warp_kernel(int N, int P, unsigned* flags, PixBatch pb, const float* __restrict__ grad_rgb,
                                     const uint8_t* __restrict__ cls, const int32_t* __restrict__ aux_probe,
                                     const float* __restrict__ aux_uv, float* __restrict__ grad_rad) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long total = pb.begin[pb.n];
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const size_t NN = (size_t)N * N;
    for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < total;
         base += warps * 32) {
        long long q = base + lane;
        bool hit = false;
        int p = -1;
        float u = 0.f, v = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
        if (q < total) {
            int lo = 0, hi = pb.n - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (pb.begin[mid] <= q) lo = mid; else hi = mid - 1;
            }
            const long long o = pb.out_offset[lo] + (q - pb.begin[lo]);
            // every pixel's saved state and gradient are valid memory: issue
            // all loads at once (one round trip), use them for HIT pixels only
            p = aux_probe[o];
            hit = cls[o] == kHit;
            u = aux_uv[2 * o];
            v = aux_uv[2 * o + 1];
            g0 = grad_rgb[3 * o];
            g1 = grad_rgb[3 * o + 1];
            g2 = grad_rgb[3 * o + 2];
            if (hit && (unsigned)p >= (unsigned)P) {  // not the saved state of a render of this grid
                atomicOr(flags, kFlagBounds);
                hit = false;
            }
        }
        int idx[4];
        float w[4] = {0.f, 0.f, 0.f, 0.f};
        if (hit) {
            bilinear_taps(N, u, v, idx, w);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int zero = 0;
                LFP_CHECK_TEXEL(flags, (unsigned)idx[k] < (unsigned)(N * N), idx[k], zero);
            }
        } else {
            g0 = g1 = g2 = 0.f;
        }
        if (__ballot_sync(full, hit) == 0u) continue;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned long long key = hit ? (unsigned long long)p * NN + (unsigned long long)idx[k] : ~0ull;
            float sx = w[k] * g0, sy = w[k] * g1, sz = w[k] * g2;
            const unsigned long long prev = __shfl_up_sync(full, key, 1);
            const unsigned long long next = __shfl_down_sync(full, key, 1);
            const unsigned heads = __ballot_sync(full, lane == 0 || key != prev);
            const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // first lane of my run
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float tx = __shfl_up_sync(full, sx, off);
                const float ty = __shfl_up_sync(full, sy, off);
                const float tz = __shfl_up_sync(full, sz, off);
                if (lane - off >= start) {
                    sx += tx;
                    sy += ty;
                    sz += tz;
                }
            }
            if (hit && (lane == 31 || next != key)) {  // last lane of a run
                float* t = grad_rad + 3 * key;
                atomicAdd(t + 0, sx);
                atomicAdd(t + 1, sy);
                atomicAdd(t + 2, sz);
            }
        }
    }
}

// Sort-by-texel adjoint: each block sorts its pixels' 4 x blockDim taps by
// texel (bitonic sort in shared memory), sums runs of equal texels and
// issues one atomic per run and channel.
constexpr int kSortThreads = 256;
constexpr int kSortTaps = 4 * kSortThreads;

__global__ void __launch_bounds__(kSortThreads) backward_sort_kernel(int N, int P, unsigned* flags, PixBatch pb,
                                                                     const float* __restrict__ grad_rgb,
                                                                     const uint8_t* __restrict__ cls,
                                                                     const int32_t* __restrict__ aux_probe,
                                                                     const float* __restrict__ aux_uv,
                                                                     float* __restrict__ grad_rad) {
    __shared__ unsigned long long s_key[kSortTaps];
    __shared__ float s_v[kSortTaps][3];
    __shared__ unsigned short s_src[kSortTaps];
    const long long total = pb.begin[pb.n];
    const size_t NN = (size_t)N * N;
    for (long long base = (long long)blockIdx.x * kSortThreads; base < total; base += (long long)gridDim.x * kSortThreads) {
        long long q = base + threadIdx.x;
        bool hit = false;
        long long o = 0;
        int p = -1;
        if (q < total) {
            int lo = 0, hi = pb.n - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (pb.begin[mid] <= q) lo = mid; else hi = mid - 1;
            }
            o = pb.out_offset[lo] + (q - pb.begin[lo]);
            p = aux_probe[o];
            hit = cls[o] == kHit;
            if (hit && (unsigned)p >= (unsigned)P) {  // not the saved state of a render of this grid
                atomicOr(flags, kFlagBounds);
                hit = false;
            }
        }
        int idx[4];
        float w[4] = {0.f, 0.f, 0.f, 0.f};
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        if (hit) {
            bilinear_taps(N, aux_uv[2 * o], aux_uv[2 * o + 1], idx, w);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int zero = 0;
                LFP_CHECK_TEXEL(flags, (unsigned)idx[k] < (unsigned)(N * N), idx[k], zero);
            }
            g0 = grad_rgb[3 * o];
            g1 = grad_rgb[3 * o + 1];
            g2 = grad_rgb[3 * o + 2];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int e = 4 * threadIdx.x + k;
            s_key[e] = hit ? (unsigned long long)p * NN + (unsigned long long)idx[k] : ~0ull;
            s_v[e][0] = w[k] * g0;
            s_v[e][1] = w[k] * g1;
            s_v[e][2] = w[k] * g2;
            s_src[e] = (unsigned short)e;
        }
        __syncthreads();
        // bitonic sort of (key, src) pairs; values follow through src
        for (int size = 2; size <= kSortTaps; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = threadIdx.x; t < kSortTaps / 2; t += kSortThreads) {
                    int a = 2 * t - (t & (stride - 1));
                    int b = a + stride;
                    bool up = (a & size) == 0;
                    unsigned long long ka = s_key[a], kb = s_key[b];
                    if ((ka > kb) == up) {
                        s_key[a] = kb;
                        s_key[b] = ka;
                        unsigned short x = s_src[a];
                        s_src[a] = s_src[b];
                        s_src[b] = x;
                    }
                }
                __syncthreads();
            }
        }
        // run heads sum their run and write it
        for (int e = threadIdx.x; e < kSortTaps; e += kSortThreads) {
            unsigned long long k = s_key[e];
            if (k == ~0ull || (e > 0 && s_key[e - 1] == k)) continue;
            float sx = 0.f, sy = 0.f, sz = 0.f;
            for (int f = e; f < kSortTaps && s_key[f] == k; ++f) {
                int src = s_src[f];
                sx += s_v[src][0];
                sy += s_v[src][1];
                sz += s_v[src][2];
            }
            float* t = grad_rad + 3 * k;
            atomicAdd(t + 0, sx);
            atomicAdd(t + 1, sy);
            atomicAdd(t + 2, sz);
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_encode_normals(const float* xyz, void* nrm, int nrm_fmt, long long n, cudaStream_t s) {
    if (nrm_fmt == kF32) encode_normals_kernel<kF32><<<blocks_for(n), kThreads, 0, s>>>(xyz, nrm, n);
    else encode_normals_kernel<kF16><<<blocks_for(n), kThreads, 0, s>>>(xyz, nrm, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_radiance(const float* rgb, void* rad, int rad_fmt, long long n, cudaStream_t s) {
    if (rad_fmt == kF32) convert_radiance_kernel<kF32><<<blocks_for(n), kThreads, 0, s>>>(rgb, rad, n);
    else convert_radiance_kernel<kF16><<<blocks_for(n), kThreads, 0, s>>>(rgb, rad, n);
    return cudaGetLastError();
}

cudaError_t launch_build_mip(const float* dist, float* mip, int count, int N, int M, cudaStream_t s) {
    long long total = (long long)count * M * M;
    build_mip_kernel<<<blocks_for(total), kThreads, 0, s>>>(dist, mip, count, N, M);
    return cudaGetLastError();
}

cudaError_t launch_build_qmin(const float* dist, float* qmin, int count, int N, cudaStream_t s) {
    build_qmin_kernel<<<count * 4, 256, 0, s>>>(dist, qmin, N);
    return cudaGetLastError();
}

cudaError_t launch_backward(int N, int P, unsigned* flags, const PixBatch& pb, const float* grad_rgb,
                            const uint8_t* cls, const int32_t* aux_probe, const float* aux_uv, float* grad_rad,
                            int reduction, cudaStream_t s) {
    long long total = pb.begin[pb.n];
    if (total == 0) return cudaSuccess;
    if (reduction == 2)
        backward_warp_kernel<<<blocks_for(total), kThreads, 0, s>>>(N, P, flags, pb, grad_rgb, cls, aux_probe, aux_uv, grad_rad);
    else if (reduction == 3)
        backward_sort_kernel<<<(int)std::min<long long>((total + kSortThreads - 1) / kSortThreads, 1 << 20),
                               kSortThreads, 0, s>>>(N, P, flags, pb, grad_rgb, cls, aux_probe, aux_uv, grad_rad);
    else
        backward_kernel<<<blocks_for(total), kThreads, 0, s>>>(N, P, flags, pb, grad_rgb, cls, aux_probe, aux_uv, grad_rad);
    return cudaGetLastError();
}

}  // namespace lfp
