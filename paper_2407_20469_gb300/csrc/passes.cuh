// passes.cuh - row and column passes of 2-D transforms on an m x m grid in
// global memory (a block's private scratch, L2-resident), staged through
// shared-memory chunks. Sparse inputs and outputs are lists of points sorted
// by (y, x) with a row-pointer array over a band of signed rows y0..y1; rows
// outside a band are never touched (they are zero on input, unneeded on output).
#pragma once

#include "fft.cuh"
#include "internal.cuh"

namespace apic {

// Bytes of dynamic shared memory for chunk buffers of one transform length N
// plus `ntw` twiddles and a 64-double reduction area.
__host__ __device__ inline size_t chunk_smem_bytes(int N, int ntw) {
    const int S = kChunk / N;
    return (size_t)2 * S * (N + 1) * sizeof(float2) + (size_t)ntw * sizeof(float2) + 64 * sizeof(double);
}

__device__ inline FFTChunk make_chunk(float2* base, int N, const float2* tw) {
    FFTChunk c;
    c.N = N;
    c.logN = ilog2(N);
    c.S = kChunk / N;                 // sequences per chunk: the most that fit and divide N
    while (c.S > 1 && N % c.S) --c.S;
    c.ld = N + 1;
    c.a = base;
    c.b = base + c.S * c.ld;
    c.tw = tw;
    return c;
}

__device__ inline void zero_smem(float2* p, int count) {
    for (int t = threadIdx.x; t < count; t += blockDim.x) p[t] = make_float2(0.f, 0.f);
}

// Builds rows y0..y1 from sparse points, transforms them along x (INV: inverse)
// and stores them into G (row index y mod m).
template <bool INV, class Val>
__device__ void rows_from_points(const FFTChunk& c, float2* G, int m, int y0, int y1, const int* rowptr,
                                 const int* px, const int* py, Val val) {
    const int ld = c.ld, lm = c.logN;
    const bool p2 = is_pow2(m);
    for (int b0 = 0; b0 <= y1 - y0; b0 += c.S) {
        const int nb = min(c.S, y1 - y0 + 1 - b0);
        zero_smem(c.a, nb * ld);
        __syncthreads();
        const int e1 = rowptr[b0 + nb];
        for (int e = rowptr[b0] + threadIdx.x; e < e1; e += blockDim.x)
            c.a[(py[e] - y0 - b0) * ld + freq_index(px[e], m)] = val(e);
        FFTChunk cc = c;
        cc.S = nb;
        const float2* R = fft_chunk<INV>(cc);
        for (int t = threadIdx.x; t < nb * m; t += blockDim.x) {
            const int s = p2 ? t >> lm : t / m, x = t - s * m;
            G[(size_t)freq_index(y0 + b0 + s, m) * m + x] = R[s * ld + x];
        }
        __syncthreads();
    }
}

// Loads rows y0..y1 of G, transforms them forward along x and hands every
// listed point's value to out(e, v).
template <class Out>
__device__ void rows_to_points(const FFTChunk& c, const float2* G, int m, int y0, int y1, const int* rowptr,
                               const int* px, const int* py, Out out) {
    const int ld = c.ld, lm = c.logN;
    const bool p2 = is_pow2(m);
    for (int b0 = 0; b0 <= y1 - y0; b0 += c.S) {
        const int nb = min(c.S, y1 - y0 + 1 - b0);
        for (int t = threadIdx.x; t < nb * m; t += blockDim.x) {
            const int s = p2 ? t >> lm : t / m, x = t - s * m;
            c.a[s * ld + x] = G[(size_t)freq_index(y0 + b0 + s, m) * m + x];
        }
        FFTChunk cc = c;
        cc.S = nb;
        const float2* R = fft_chunk<false>(cc);
        const int e1 = rowptr[b0 + nb];
        for (int e = rowptr[b0] + threadIdx.x; e < e1; e += blockDim.x)
            out(e, R[(py[e] - y0 - b0) * ld + freq_index(px[e], m)]);
        __syncthreads();
    }
}

// For every column of G: rows yi0..yi1 are the input (others zero), inverse
// transform along y, mid(R, c0) edits the values R[s * ld + y] of columns
// c0 + s, forward transform along y, rows yo0..yo1 are stored back.
template <class Mid>
__device__ void cols_inv_mid_fwd(const FFTChunk& c, float2* G, int m, int yi0, int yi1, int yo0, int yo1, Mid mid) {
    const int ld = c.ld, S = c.S;
    const int nbi = yi1 - yi0 + 1, nbo = yo1 - yo0 + 1;
    for (int c0 = 0; c0 < m; c0 += S) {
        zero_smem(c.a, S * ld);
        __syncthreads();
        for (int t = threadIdx.x; t < nbi * S; t += blockDim.x) {
            const int b = t / S, s = t - b * S;
            const int y = freq_index(yi0 + b, m);
            c.a[s * ld + y] = G[(size_t)y * m + c0 + s];
        }
        float2* R = fft_chunk<true>(c);
        mid(R, c0);
        FFTChunk c2 = c;
        c2.a = R;
        c2.b = (R == c.a) ? c.b : c.a;
        const float2* R2 = fft_chunk<false>(c2);
        for (int t = threadIdx.x; t < nbo * S; t += blockDim.x) {
            const int b = t / S, s = t - b * S;
            const int y = freq_index(yo0 + b, m);
            G[(size_t)y * m + c0 + s] = R2[s * ld + y];
        }
        __syncthreads();
    }
}

}  // namespace apic
