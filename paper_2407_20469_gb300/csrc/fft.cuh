// fft.cuh - batched complex FFTs (power-of-two lengths, and 3 times a power of two)
// of a chunk of sequences held in shared memory, computed by all threads of a block.
//
// Layout: S sequences of length N, sequence s at a + s * ld (ld >= N, chosen
// odd so that column-wise staging is bank-conflict free). Each stage is a
// Stockham radix-4 step (natural order in, natural order out, ping-pong between
// buffers a and b); an odd log2(N) ends with one radix-2 step. The twiddle
// table holds W^k = exp(-2 pi i k / N), k < N; the inverse transform uses the
// conjugates and is unnormalised (sum_k X_k exp(+2 pi i k n / N)).
#pragma once

#include "common.cuh"

namespace apic {

struct FFTChunk {
    float2* a;          // S * ld
    float2* b;          // S * ld (ping-pong)
    const float2* tw;   // N twiddles
    int N, logN, S, ld;
};

template <bool INV>
__device__ __forceinline__ float2 twiddle(const float2* tw, int k) {
    const float2 w = tw[k];
    return INV ? make_float2(w.x, -w.y) : w;
}

template <bool INV>
__device__ __forceinline__ void radix4(float2& v0, float2& v1, float2& v2, float2& v3) {
    const float2 t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3);
    const float2 d = csub(v1, v3);
    // forward: t3 = -i d ; inverse: t3 = +i d
    const float2 t3 = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
    v0 = cadd(t0, t2);
    v2 = csub(t0, t2);
    v1 = cadd(t1, t3);
    v3 = csub(t1, t3);
}

__host__ __device__ inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// One Stockham step of radix R (2, 3 or 4) on every sequence of the chunk, for any
// length N divisible by Ns R (index arithmetic by division): inputs x[j + r N / R],
// j < N / R, k = j mod Ns, twiddled by W^(r k N / (Ns R)) (W = exp(-2 pi i / N), the
// chunk's table), a DFT_R, outputs at (j - k) R + k + r Ns.
template <int R, bool INV>
__device__ void stockham_step(const float2* src, float2* dst, const FFTChunk& c, int Ns) {
    const int N = c.N, ld = c.ld, q = N / R, total = c.S * q, tstep = N / (Ns * R);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int s = t / q, j = t - s * q, k = j % Ns;
        const float2* in = src + s * ld;
        float2* out = dst + s * ld;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            v[r] = in[j + r * q];
            if (r > 0 && k) v[r] = cmul(v[r], twiddle<INV>(c.tw, r * k * tstep));
        }
        if constexpr (R == 2) {
            const float2 a = v[0], b = v[1];
            v[0] = cadd(a, b);
            v[1] = csub(a, b);
        } else if constexpr (R == 4) {
            radix4<INV>(v[0], v[1], v[2], v[3]);
        } else {
            // X1,2 = a0 - (a1 + a2) / 2 -/+ i (sqrt(3) / 2)(a1 - a2) (forward; the inverse flips the sign of i)
            const float h = 0.86602540378443865f;
            const float2 sm = cadd(v[1], v[2]), d = csub(v[1], v[2]);
            const float2 m = make_float2(v[0].x - 0.5f * sm.x, v[0].y - 0.5f * sm.y);
            const float2 rr = INV ? make_float2(-h * d.y, h * d.x) : make_float2(h * d.y, -h * d.x);
            v[0] = cadd(v[0], sm);
            v[1] = cadd(m, rr);
            v[2] = csub(m, rr);
        }
        const int o = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[o + r * Ns] = v[r];
    }
    __syncthreads();
}

// Transforms of length N = 3 * 2^k (output grids with 3x upsampling): a radix-3 step,
// then radix-4 steps and, for an odd power of two, a radix-2 step.
template <bool INV>
__device__ float2* fft_chunk_3(const FFTChunk& c) {
    float2* src = c.a;
    float2* dst = c.b;
    __syncthreads();
    int Ns = 1;
    stockham_step<3, INV>(src, dst, c, Ns);
    Ns *= 3;
    float2* t = src;
    src = dst;
    dst = t;
    while (Ns * 4 <= c.N) {
        stockham_step<4, INV>(src, dst, c, Ns);
        Ns *= 4;
        t = src;
        src = dst;
        dst = t;
    }
    if (Ns < c.N) {
        stockham_step<2, INV>(src, dst, c, Ns);
        t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// Transforms every sequence of the chunk in c.a; returns the buffer holding
// the result (c.a or c.b). Starts and ends with __syncthreads. N a power of two,
// or 3 times one (fft_chunk_3).
template <bool INV>
__device__ float2* fft_chunk(const FFTChunk& c) {
    if (!is_pow2(c.N)) return fft_chunk_3<INV>(c);
    float2* src = c.a;
    float2* dst = c.b;
    const int N = c.N, ld = c.ld;
    const int q4 = N >> 2, lq4 = c.logN - 2;
    __syncthreads();
    int Ns = 1, lNs = 0;
    for (int st = 0; st < (c.logN >> 1); ++st) {
        const int total = c.S << lq4;
        const int twshift = c.logN - lNs - 2;  // N / (4 Ns) = 2^twshift
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int s = t >> lq4, j = t & (q4 - 1);
            const float2* in = src + s * ld;
            float2* out = dst + s * ld;
            const int k = j & (Ns - 1);
            float2 v0 = in[j], v1 = in[j + q4], v2 = in[j + 2 * q4], v3 = in[j + 3 * q4];
            if (k) {
                const int e = k << twshift;
                v1 = cmul(v1, twiddle<INV>(c.tw, e));
                v2 = cmul(v2, twiddle<INV>(c.tw, 2 * e));
                v3 = cmul(v3, twiddle<INV>(c.tw, 3 * e));
            }
            radix4<INV>(v0, v1, v2, v3);
            const int o = ((j - k) << 2) + k;
            out[o] = v0;
            out[o + Ns] = v1;
            out[o + 2 * Ns] = v2;
            out[o + 3 * Ns] = v3;
        }
        __syncthreads();
        float2* t2 = src;
        src = dst;
        dst = t2;
        Ns <<= 2;
        lNs += 2;
    }
    if (c.logN & 1) {
        const int q2 = N >> 1, lq2 = c.logN - 1;
        const int total = c.S << lq2;
        const int twshift = c.logN - lNs - 1;  // N / (2 Ns)
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int s = t >> lq2, j = t & (q2 - 1);
            const float2* in = src + s * ld;
            float2* out = dst + s * ld;
            const int k = j & (Ns - 1);
            float2 v0 = in[j], v1 = in[j + q2];
            if (k) v1 = cmul(v1, twiddle<INV>(c.tw, k << twshift));
            const int o = ((j - k) << 1) + k;
            out[o] = cadd(v0, v1);
            out[o + Ns] = csub(v0, v1);
        }
        __syncthreads();
        float2* t2 = src;
        src = dst;
        dst = t2;
    }
    return src;
}

// Copies N twiddles from global memory into shared memory.
__device__ __forceinline__ void load_twiddles(float2* s_tw, const float2* g_tw, int N) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) s_tw[i] = g_tw[i];
}

__host__ __device__ inline int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

}  // namespace apic
