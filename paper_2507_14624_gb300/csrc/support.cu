// Upload-time conversions, the min/max low-resolution map and the adjoint.
#include <cuda_runtime.h>

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
__global__ void build_mip_kernel(const float* __restrict__ dist, float2* __restrict__ mip, int count, int N, int M) {
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
        mip[c] = make_float2(lo, hi);
    }
}

// Adjoint: for every HIT pixel add w_k * g_c into the 4 bilinear taps.
__global__ void backward_kernel(int N, PixBatch pb, const float* __restrict__ grad_rgb,
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
        if (p < 0) continue;
        int idx[4];
        float w[4];
        bilinear_taps(N, aux_uv[2 * o], aux_uv[2 * o + 1], idx, w);
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

cudaError_t launch_build_mip(const float* dist, float2* mip, int count, int N, int M, cudaStream_t s) {
    long long total = (long long)count * M * M;
    build_mip_kernel<<<blocks_for(total), kThreads, 0, s>>>(dist, mip, count, N, M);
    return cudaGetLastError();
}

cudaError_t launch_backward(int N, const PixBatch& pb, const float* grad_rgb, const uint8_t* cls,
                            const int32_t* aux_probe, const float* aux_uv, float* grad_rad, cudaStream_t s) {
    long long total = pb.begin[pb.n];
    if (total == 0) return cudaSuccess;
    backward_kernel<<<blocks_for(total), kThreads, 0, s>>>(N, pb, grad_rgb, cls, aux_probe, aux_uv, grad_rad);
    return cudaGetLastError();
}

}  // namespace lfp
