// common.cuh - small device helpers shared by the kernels of this library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace apic {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

// Signed frequency of DFT index i on an n-point axis (Nyquist -> -n/2).
__device__ __forceinline__ int signed_freq(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }
// DFT index of signed frequency k on an n-point axis.
__device__ __forceinline__ int freq_index(int k, int n) {
    int r = k % n;
    return r < 0 ? r + n : r;
}

// Wraps an angle into [-pi, pi).
__device__ __forceinline__ float wrap_pi(float a) {
    const float two_pi = 6.283185307179586f;
    return a - two_pi * floorf((a + 3.14159265358979f) * 0.15915494309189535f);
}

// Block-wide sum of doubles; `red` holds >= 32 doubles of shared memory.
// Every thread gets the total. Contains __syncthreads.
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0;
    for (int i = 0; i < nw; ++i) t += red[i];
    __syncthreads();
    return t;
}

// Block-wide sum of doubles. Warps reduce with shuffles, warp 0 combines the
// warp partials and broadcasts the total, so each thread does five FP64 adds
// rather than one per warp. `red` holds 64 doubles; the caller alternates
// `parity` (0/1) between consecutive calls so that partials of one call are
// never overwritten while another warp is still reading them.
__device__ __forceinline__ double block_sum2(double v, double* red, int& parity) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    double* r = red + parity * 32;
    if (lane == 0) r[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? r[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) r[31] = t;
    }
    __syncthreads();
    const double total = r[31];
    parity ^= 1;
    return total;
}

// block_sum2 of FP32 per-thread partials: FP32 within each warp, FP64 across the
// warps (a handful of FP64 adds on warp 0 instead of five per lane of every warp).
__device__ __forceinline__ double block_sum2f(float v, double* red, int& parity) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    double* r = red + parity * 32;
    if (lane == 0) r[warp] = (double)v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? r[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) r[31] = t;
    }
    __syncthreads();
    const double total = r[31];
    parity ^= 1;
    return total;
}

// Raises (never lowers) a kernel's dynamic shared-memory limit. The limit is
// process-wide per function, so plans of different sizes that share a kernel
// must not shrink it under one another.
inline cudaError_t raise_smem_limit(const void* f, size_t smem) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, f);
    if (e != cudaSuccess) return e;
    if ((size_t)a.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace apic
