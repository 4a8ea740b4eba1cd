// kernels_peak.cu - measured FMA throughput of the device's CUDA cores (FP32 and
// FP64), the denominators of the rooflines of the ALU-bound stages.
//
// Every thread runs kChains independent multiply-add chains a <- a b + c for
// `iters` steps (kChains chains hide the FMA latency); the chains' sum is stored
// only under a condition that never holds, so nothing is optimised away and the
// kernel writes no memory. Rate = 2 kChains iters threads / event time.
#include <cuda_runtime.h>

#include "../../include/apic.h"
#include "internal.cuh"

namespace apic {

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <class T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_rate(T* out, int iters, T b, T c) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (out && s == (T)-1.2345e30) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true: out is NULL
}

template <class T>
cudaError_t rate(int iters, double* flops_per_s) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate<T>, kPeakThreads, 0);
    if (e != cudaSuccess) return e;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    // b slightly below 1 and c small keep every chain finite and away from denormals
    const T b = (T)0.999999, c = (T)1e-6;
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {      // first launch is the warm-up
        cudaEventRecord(e0, 0);
        k_fma_rate<T><<<blocks, kPeakThreads, 0, 0>>>(nullptr, iters, b, c);
        cudaEventRecord(e1, 0);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    *flops_per_s = 2.0 * kChains * (double)iters * blocks * kPeakThreads / (best * 1e-3);
    return cudaSuccess;
}

}  // namespace

cudaError_t measure_fma_rate(int precision, double* flops_per_s) {
    if (precision == 32) return rate<float>(1 << 16, flops_per_s);
    if (precision == 64) return rate<double>(1 << 11, flops_per_s);
    return cudaErrorInvalidValue;
}

}  // namespace apic
