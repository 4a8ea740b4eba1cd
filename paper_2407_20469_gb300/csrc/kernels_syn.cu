// kernels_syn.cu - final inverse transform of the stitched spectrum onto the
// upsampled grid, and the forward model (Eq. 1-2) used to synthesise inputs.
#include <math.h>

#include "../../include/apic.h"
#include "passes.cuh"
#include "regfft.cuh"

namespace apic {

// ---------------------------------------------------------------- synthesis
// field(x) = sum_K O(K) exp(2 pi i K.x / N) on the N x N output grid; the output
// buffer is the transform's scratch. Rows of the aperture band are built from
// the sparse spectrum, then every column is inverse-transformed along y.
__global__ void __launch_bounds__(kThreads) k_synthesize(DevPlan P, int n_tiles, const float2* __restrict__ spec,
                                                         float2* __restrict__ field,
                                                         const int32_t* __restrict__ status) {
    extern __shared__ float4 smem4[];
    float2* sm = reinterpret_cast<float2*>(smem4);
    const int N = P.H;
    float2* tw = sm + 2 * (kChunk / N) * (N + 1);
    load_twiddles(tw, P.tw_N, N);
    const FFTChunk c = make_chunk(sm, N, tw);
    const int S = c.S, ld = c.ld;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        float2* F = field + (size_t)tile * N * N;
        if (status && (status[tile] & (APIC_TILE_BACKGROUND | APIC_TILE_BADINPUT))) {
            for (size_t t = threadIdx.x; t < (size_t)N * N; t += blockDim.x) F[t] = make_float2(0.f, 0.f);
            continue;
        }
        const float2* sp = spec + (size_t)tile * P.nap;
        rows_from_points<true>(c, F, N, P.ap_y0, P.ap_y1, P.ap_rowptr, P.ap_x, P.ap_y,
                               [&](int e) { return sp[e]; });
        const int nb = P.ap_y1 - P.ap_y0 + 1;
        for (int c0 = 0; c0 < N; c0 += S) {
            zero_smem(c.a, S * ld);
            __syncthreads();
            for (int t = threadIdx.x; t < nb * S; t += blockDim.x) {
                const int b = t / S, q = t - b * S;
                const int y = freq_index(P.ap_y0 + b, N);
                c.a[q * ld + y] = F[(size_t)y * N + c0 + q];
            }
            const float2* R = fft_chunk<true>(c);
            for (int t = threadIdx.x; t < S * N; t += blockDim.x) {   // final values: evict first from L2
                const int y = t / S, q = t - y * S;
                __stcs(F + (size_t)y * N + c0 + q, R[q * ld + y]);
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------- synthesis, register transforms
// The same sum for output sides N = 32 B (B = 16, 32: 512 and 1024), one block of 16 warps
// per tile (persistent over tiles), each warp transforming one N-point sequence at a time
// in registers: lane t holds x[t + 32 j] (j < B); step A a DFT_B in registers, the twiddle
// W_N^(t k2) and a padded shared-memory transpose, step B lanes k2 < B run a DFT_32, so
// lane k2 ends with X[k2 + B k1] (k1 < 32). Columns first, rows last, so that the final
// writes are whole rows:
//   1 columns x of the aperture (ap_x0..ap_x1, in groups of 16, one per warp): the
//     column's points (list sorted by (x, y)) scattered into the warp's area, inverse
//     transform along y; the 16 columns staged through shared memory (half the rows at
//     a time) and stored as 128-byte row segments into the tile's own output rows at
//     columns 0..ap_x1 - ap_x0 (the output buffer is the scratch);
//   2 every row: its aperture columns loaded, the rest zero, inverse transform along x,
//     the row stored whole (evict-first).
constexpr int kSRWarps = 16;
constexpr int kSRLd = 33;            // a warp's area: 32 rows of 33 values (the scatter uses N of them)

template <int B>
__device__ __forceinline__ void warp_fft_inv(float2 (&v)[B], float2 (&o)[32], float2* hs, const float2* tw, int lane) {
    DFT<B, true>::run(v);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) hs[k2 * kSRLd + lane] = cmul(v[k2], tw_get(tw, k2 * 32 + lane, true));
    __syncwarp();
    const int row = lane < B ? lane : 0;          // lanes k2 >= B transform a copy, discarded
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) o[n1] = hs[row * kSRLd + n1];
    DFT<32, true>::run(o);
    __syncwarp();
}

size_t synr_smem_bytes(int H) {
    return (size_t)kSRWarps * 32 * kSRLd * sizeof(float2) + (size_t)H * sizeof(float2);
}

template <int B>
__global__ void __launch_bounds__(kSRWarps * 32, 1)
k_synth_reg(DevPlan P, int n_tiles, const float2* __restrict__ spec, float2* __restrict__ field,
            const int32_t* __restrict__ status) {
    constexpr int N = 32 * B, HALF = N / 2;
    extern __shared__ float4 smem4[];
    float2* areas = reinterpret_cast<float2*>(smem4);
    float2* tw = areas + kSRWarps * 32 * kSRLd;     // [k2 < B][t < 32] = W_N^(t k2)
    float2* stage = areas;                          // HALF x 17 values, aliases the warps' areas
    for (int i = threadIdx.x; i < 32 * B; i += blockDim.x) {
        const int k2 = i >> 5, t = i & 31;
        tw[i] = P.tw_N[(t * k2) % N];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* hs = areas + warp * 32 * kSRLd;
    const int x0 = P.ap_x0, nbx = P.ap_x1 - P.ap_x0 + 1;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        float2* F = field + (size_t)tile * N * N;
        if (status && (status[tile] & (APIC_TILE_BACKGROUND | APIC_TILE_BADINPUT))) {
            for (size_t t = threadIdx.x; t < (size_t)N * N; t += blockDim.x) F[t] = make_float2(0.f, 0.f);
            continue;
        }
        const float2* sp = spec + (size_t)tile * P.nap;
        // 1: aperture columns, 16 at a time
        for (int c0 = 0; c0 < nbx; c0 += kSRWarps) {
            const int c = c0 + warp;
            float2 o[32];
            if (c < nbx) {
#pragma unroll
                for (int j = 0; j < B; ++j) hs[lane + 32 * j] = make_float2(0.f, 0.f);
                __syncwarp();
                for (int e = P.ap_colptr[c] + lane; e < P.ap_colptr[c + 1]; e += 32) {
                    const int p = P.ap_cole[e];
                    hs[freq_index(P.ap_y[p], N)] = sp[p];
                }
                __syncwarp();
                float2 v[B];
#pragma unroll
                for (int j = 0; j < B; ++j) v[j] = hs[lane + 32 * j];
                __syncwarp();
                warp_fft_inv<B>(v, o, hs, tw, lane);   // lane k2 < B: rows k2 + B k1
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                __syncthreads();                        // areas free (h = 0) / stage consumed (h = 1)
                if (c < nbx && lane < B) {
#pragma unroll
                    for (int k1 = 16 * h; k1 < 16 * h + 16; ++k1) stage[(lane + B * k1 - h * HALF) * 17 + warp] = o[k1];
                }
                __syncthreads();
                const int ncol = min(kSRWarps, nbx - c0);
                for (int i = threadIdx.x; i < HALF * kSRWarps; i += blockDim.x) {
                    const int y = i >> 4, q = i & 15;
                    if (q < ncol) F[(size_t)(h * HALF + y) * N + c0 + q] = stage[y * 17 + q];
                }
            }
            __syncthreads();                            // stage consumed before the areas are reused
        }
        // 2: rows (each warp reads its own rows' aperture columns before overwriting them)
        for (int y = warp; y < N; y += kSRWarps) {
            float2* row = F + (size_t)y * N;
            float2 v[B], o[32];
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const int x = lane + 32 * j;
                const int c = (x < N / 2 ? x : x - N) - x0;
                v[j] = (unsigned)c < (unsigned)nbx ? row[c] : make_float2(0.f, 0.f);
            }
            warp_fft_inv<B>(v, o, hs, tw, lane);
            if (lane < B) {
#pragma unroll
                for (int k1 = 0; k1 < 32; ++k1) __stcs(row + lane + B * k1, o[k1]);
            }
        }
        __syncthreads();
    }
}

template <int B>
static int configure_synr_b(size_t smem) {
    if (raise_smem_limit((const void*)k_synth_reg<B>, smem) != cudaSuccess) return 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_synth_reg<B>, kSRWarps * 32, smem) != cudaSuccess)
        return 0;
    return occ;
}

int configure_synr(int H, size_t smem) {
    if (H == 512) return configure_synr_b<16>(smem);
    if (H == 1024) return configure_synr_b<32>(smem);
    return 0;
}

cudaError_t launch_synthesize(const DevPlan& P, const Launch& L, int n_tiles, const float2* spec, float2* field,
                              const int32_t* status, cudaStream_t st) {
    if (L.grid_synr > 0 && (P.H == 512 || P.H == 1024)) {
        const int grid = min(L.grid_synr, n_tiles);
        if (grid < 1) return cudaSuccess;
        if (P.H == 512)
            k_synth_reg<16><<<grid, kSRWarps * 32, L.smem_synr, st>>>(P, n_tiles, spec, field, status);
        else
            k_synth_reg<32><<<grid, kSRWarps * 32, L.smem_synr, st>>>(P, n_tiles, spec, field, status);
        return cudaGetLastError();
    }
    const int grid = min(L.grid_syn, n_tiles);
    k_synthesize<<<grid, kThreads, L.smem_syn, st>>>(P, n_tiles, spec, field, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- simulator
// Counter-based uniform numbers: the SplitMix64 output function (Steele, Lea
// and Flood, 2014) applied to seed + counter * golden-ratio increment.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
struct Rng {
    unsigned long long key, ctr;
    __device__ float uniform() {  // in (0, 1)
        const unsigned long long z = mix64(key + (++ctr) * 0x9E3779B97F4A7C15ull);
        return ((float)(z >> 40) + 0.5f) * (1.0f / 16777216.0f);
    }
};

// Poisson variate: multiplication method for lam < 10, otherwise the
// transformed rejection with squeeze "PTRS" of Hoermann (1993). The number of
// trials is bounded; on exhaustion the rounded mean is returned.
__device__ float poisson(float lam, Rng& g) {
    if (!(lam > 0.f)) return 0.f;
    if (lam < 10.f) {
        const float L = expf(-lam);
        float p = 1.f;
        int k = 0;
        for (; k < 200; ++k) {
            p *= g.uniform();
            if (p <= L) break;
        }
        return (float)k;
    }
    const float slam = sqrtf(lam), loglam = logf(lam);
    const float b = 0.931f + 2.53f * slam;
    const float a = -0.059f + 0.02483f * b;
    const float inv_alpha = 1.1239f + 1.1328f / (b - 3.4f);
    const float vr = 0.9277f - 3.6224f / (b - 2.f);
    for (int trial = 0; trial < 64; ++trial) {
        const float U = g.uniform() - 0.5f;
        const float V = g.uniform();
        const float us = 0.5f - fabsf(U);
        const float k = floorf((2.f * a / us + b) * U + lam + 0.43f);
        if (us >= 0.07f && V <= vr) return k;
        if (k < 0.f || (us < 0.013f && V > us)) continue;
        if (logf(V) + logf(inv_alpha) - logf(a / (us * us) + b) <= -lam + k * loglam - lgammaf(k + 1.f)) return k;
    }
    return rintf(lam);
}

// Object spectrum O = DFT(o) / (N N), one tile per block (persistent).
__global__ void __launch_bounds__(kThreads) k_sim_object(DevPlan P, int n_tiles, const float2* __restrict__ obj,
                                                         float2* __restrict__ ohat) {
    extern __shared__ float4 smem4[];
    float2* sm = reinterpret_cast<float2*>(smem4);
    const int N = P.H, lN = ilog2(N);
    const bool p2 = is_pow2(N);
    float2* tw = sm + 2 * (kChunk / N) * (N + 1);
    load_twiddles(tw, P.tw_N, N);
    const FFTChunk c = make_chunk(sm, N, tw);
    const int S = c.S, ld = c.ld;
    const float scale = 1.f / ((float)N * (float)N);
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const float2* o = obj + (size_t)tile * N * N;
        float2* O = ohat + (size_t)tile * N * N;
        for (int r0 = 0; r0 < N; r0 += S) {
            for (int t = threadIdx.x; t < S * N; t += blockDim.x) {
                const int q = p2 ? t >> lN : t / N, x = t - q * N;
                c.a[q * ld + x] = o[(size_t)(r0 + q) * N + x];
            }
            const float2* R = fft_chunk<false>(c);
            for (int t = threadIdx.x; t < S * N; t += blockDim.x) {
                const int q = p2 ? t >> lN : t / N, x = t - q * N;
                O[(size_t)(r0 + q) * N + x] = R[q * ld + x];
            }
            __syncthreads();
        }
        for (int c0 = 0; c0 < N; c0 += S) {
            for (int t = threadIdx.x; t < S * N; t += blockDim.x) {
                const int y = t / S, q = t - y * S;
                c.a[q * ld + y] = O[(size_t)y * N + c0 + q];
            }
            const float2* R = fft_chunk<false>(c);
            for (int t = threadIdx.x; t < S * N; t += blockDim.x) {
                const int y = t / S, q = t - y * S;
                O[(size_t)y * N + c0 + q] = cscale(R[q * ld + y], scale);
            }
            __syncthreads();
        }
    }
}

// Intensity of image i of a tile: S_i(k) = O(k - k_i) exp(j phi(k)) on the
// pupil (Eq. 1), I_i = |IDFT(S_i)|^2 (Eq. 2), optional Poisson noise.
// One (tile, image) per block (persistent); scratch n x n per block.
__global__ void __launch_bounds__(kThreads) k_sim_images(DevPlan P, int n_tiles, const float2* __restrict__ ohat,
                                                         const float* __restrict__ phi, float photons,
                                                         unsigned long long seed, float* __restrict__ I,
                                                         float2* __restrict__ scratch) {
    extern __shared__ float4 smem4[];
    float2* sm = reinterpret_cast<float2*>(smem4);
    const int n = P.h, N = P.H;
    float2* tw = sm + 2 * (kChunk / n) * (n + 1);
    load_twiddles(tw, P.tw_n, n);
    const FFTChunk c = make_chunk(sm, n, tw);
    const int S = c.S, ld = c.ld;
    float2* G = scratch + (size_t)blockIdx.x * n * n;
    const int nprob = n_tiles * P.n_img;
    for (int prob = blockIdx.x; prob < nprob; prob += gridDim.x) {
        const int tile = prob / P.n_img, i = prob - tile * P.n_img;
        const float2* O = ohat + (size_t)tile * N * N;
        const float* ph = phi + (size_t)tile * P.npup;
        const int kix = P.led_x[i], kiy = P.led_y[i];
        rows_from_points<true>(c, G, n, -P.pup_ay, P.pup_ay, P.pup_rowptr, P.pup_x, P.pup_y, [&](int e) {
            const int Kx = P.pup_x[e] - kix, Ky = P.pup_y[e] - kiy;
            float sn, cs;
            sincosf(ph[e], &sn, &cs);
            return cmul(O[(size_t)freq_index(Ky, N) * N + freq_index(Kx, N)], make_float2(cs, sn));
        });
        float* img = I + ((size_t)tile * P.n_img + i) * n * n;
        const int nb = 2 * P.pup_ay + 1;
        for (int c0 = 0; c0 < n; c0 += S) {
            zero_smem(c.a, S * ld);
            __syncthreads();
            for (int t = threadIdx.x; t < nb * S; t += blockDim.x) {
                const int b = t / S, q = t - b * S;
                const int y = freq_index(-P.pup_ay + b, n);
                c.a[q * ld + y] = G[(size_t)y * n + c0 + q];
            }
            const float2* R = fft_chunk<true>(c);
            for (int t = threadIdx.x; t < S * n; t += blockDim.x) {
                const int y = t / S, q = t - y * S;
                float v = cabs2(R[q * ld + y]);
                if (photons > 0.f) {
                    Rng g{seed ^ mix64(((unsigned long long)prob << 32) | (unsigned)(y * n + c0 + q)), 0ull};
                    v = poisson(v * photons, g) / photons;
                }
                img[(size_t)y * n + c0 + q] = v;
            }
            __syncthreads();
        }
    }
}

cudaError_t launch_sim(const DevPlan& P, const Launch& L, int n_tiles, const float2* obj, const float* phi,
                       float photons, unsigned long long seed, float* I, float2* ohat_scratch, cudaStream_t st) {
    // ohat_scratch: n_tiles * H * H complex, followed by grid_sim * h * h complex
    const int g1 = min(L.grid_syn, n_tiles);
    k_sim_object<<<g1, kThreads, L.smem_syn, st>>>(P, n_tiles, obj, ohat_scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float2* G = ohat_scratch + (size_t)n_tiles * P.H * P.H;
    const int g2 = min(L.grid_sim, n_tiles * P.n_img);
    k_sim_images<<<g2, kThreads, L.smem_sim, st>>>(P, n_tiles, ohat_scratch, phi, photons, seed, I, G);
    return cudaGetLastError();
}

}  // namespace apic
