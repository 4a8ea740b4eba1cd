// kernels_kkr.cu - Kramers-Kronig recovery (WSI-APIC Eq. 4-7) with
// register-resident half-warp FFTs (n = 16 BN; BN = 32 for 512-pixel tiles uses the
// wide form, two step-B rows per lane).
//
// One block per (tile, NA-matching image) problem, persistent over problems;
// an n x n complex scratch grid per block (L2-resident; HBM at n = 512), stored in
// 4 x 4 tiles (t4grid.cuh) so that the column passes move whole sectors. Each
// half-warp transforms one row or column at a time:
//   P1 rows: log(max(I, 1e-6 mean I)), forward transform along x
//   P2 cols: forward along y, half-plane mask of Eq. 5, inverse along y
//   P3 rows: inverse along x, / n^2, exp (Eq. 6), forward along x; only the
//            columns the gather needs (the pupil box shifted by -k_i) are kept
//   P4 cols: those columns forward along y, / n^2 (Fourier-series
//            coefficients, Eq. 7), rows of the shifted pupil box kept
// then the values at K = k_p - k_i for the pupil points k_p are gathered.
// log, exp and sincos are the hardware approximations (__logf, __expf,
// __sincosf): their errors (a few 1e-7 relative for the log-intensities and
// amplitudes here, ~1e-6 absolute for phases of a few radians) sit far below
// the 2e-4 spectrum tolerance the tests hold, and the accurate versions' slow
// paths cost this kernel 30 % of its time (instruction-fetch stalls).
#include <math.h>

#include "../../include/apic.h"
#include "internal.cuh"
#include "regfft.cuh"
#include "t4grid.cuh"

namespace apic {

namespace {

constexpr int kKKThreads = 512;
constexpr int kKKHW = kKKThreads / 16;

__device__ __forceinline__ int sfreq_kk(int i, int n) { return i < n / 2 ? i : i - n; }

}  // namespace

size_t kkr_smem_bytes(int BN) {
    const int hws = hw_single_size(BN);
    return (size_t)kKKHW * hws * sizeof(float2) + (size_t)2 * 16 * BN * sizeof(float2) + 64 * sizeof(double);
}

template <int BN>
__global__ void __launch_bounds__(kKKThreads, 1)
k_kk_reg(DevPlan P, int n_tiles, const float* __restrict__ I, float2* __restrict__ xdisc, float2* __restrict__ scratch,
         const int32_t* __restrict__ status) {
    constexpr int n = 16 * BN, HWS = HWSize<BN>::value, S = Slots<BN>::value;
    extern __shared__ float4 smem4[];
    float2* hw_area = reinterpret_cast<float2*>(smem4);
    float2* tw = hw_area + kKKHW * HWS;
    double* red = reinterpret_cast<double*>(tw + 2 * n);
    make_step_twiddles(tw, P.tw_n, BN);
    __syncthreads();

    const int hw = threadIdx.x >> 4, t = threadIdx.x & 15;
    const HalfWarp h{t, (threadIdx.x & 16) ? 0xFFFF0000u : 0x0000FFFFu, hw_area + hw * HWS};
    float2* G = scratch + (size_t)blockIdx.x * n * n;
    const T4Lane L(t);
    const int lrow = t4_row(t, n), lcol = t4_col(t);      // this lane's row / column offsets
    const float inv_n2 = 1.0f / (float)(n * n);
    const long long hh = (long long)P.h * P.h, ww = (long long)P.w * P.w;
    const int nprob = n_tiles * P.n_bf;

    int par = 0;
    for (int prob = blockIdx.x; prob < nprob; prob += gridDim.x) {
        const int tile = prob / P.n_bf, i = prob - tile * P.n_bf;
        if (status && (status[tile] & (APIC_TILE_BACKGROUND | APIC_TILE_BADINPUT))) continue;
        const float* img = I + ((size_t)tile * P.n_img + i) * n * n;
        const int kix = P.led_x[i], kiy = P.led_y[i];
        // image sum for the log floor: FP32 within a thread (n^2 / 512 values) and a warp
        float s = 0.f;
        const float4* img4 = reinterpret_cast<const float4*>(img);
        for (int q = threadIdx.x; q < n * n / 4; q += blockDim.x) {
            const float4 v = img4[q];
            s += (v.x + v.y) + (v.z + v.w);
        }
        const double stot = block_sum2f(s, red, par);
        const float eps = (float)(1e-6 * stot / ((double)n * n));

        // P1: rows, log then forward along x
        for (int r = hw; r < n; r += kKKHW) {
            const float* row = img + (size_t)r * n;
            float2 v[BN], o[S][16];
#pragma unroll
            for (int j = 0; j < BN; ++j)      // last read of the image: evict first from L2
                v[j] = make_float2(__logf(fmaxf(__ldcs(row + t + 16 * j), eps)), 0.f);
            fft_a<BN, false>(v, o, h, tw);
            float2* gr = G + t4_row(r, n);
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (t + 16 * s < BN) {
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) gr[L.at(16 * s + BN * k1)] = o[s][k1];
                }
        }
        __syncthreads();
        // P2: columns, forward along y, Eq. 5 mask, inverse along y
        for (int x = hw; x < n; x += kKKHW) {
            float2 v[BN], o[S][16];
            float2* gc = G + lrow + t4_col(x);              // rows t + 16 j of column x
#pragma unroll
            for (int j = 0; j < BN; ++j) v[j] = gc[16 * j * n];
            fft_a<BN, false>(v, o, h, tw);
            const long long kxp = (long long)sfreq_kk(x, n) * kix * hh;
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (t + 16 * s < BN) {
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) {
                        const long long dot = kxp + (long long)sfreq_kk(t + 16 * s + BN * k1, n) * kiy * ww;
                        const float f = dot < 0 ? 1.f : (dot == 0 ? 0.5f : 0.f);
                        o[s][k1] = cscale(o[s][k1], f);
                    }
                }
            fft_b<BN, true>(o, v, h, tw);
#pragma unroll
            for (int k1 = 0; k1 < BN; ++k1) gc[16 * k1 * n] = v[k1];
        }
        __syncthreads();
        // only the spectrum at K = k_p - k_i (|k_p| within the pupil box) is gathered:
        // columns Kx in [kx0, kx0 + nbx), rows Ky in [ky0, ky0 + nby)
        const int kx0 = -P.pup_ax - kix, nbx = 2 * P.pup_ax + 1;
        const int ky0 = -P.pup_ay - kiy, nby = 2 * P.pup_ay + 1;
        // P3: rows, inverse along x, exp, forward along x; the band columns are stored
        for (int r = hw; r < n; r += kKKHW) {
            float2* gr = G + t4_row(r, n) + lcol;           // columns t + 16 j of row r
            float2 v[BN], o[S][16];
#pragma unroll
            for (int j = 0; j < BN; ++j) v[j] = gr[64 * j];
            fft_a<BN, true>(v, o, h, tw);
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (t + 16 * s < BN) {
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) {
                        const float2 z = cscale(o[s][k1], inv_n2);
                        float sn, cs;
                        __sincosf(z.y, &sn, &cs);
                        const float e = __expf(z.x);
                        o[s][k1] = make_float2(e * cs, e * sn);
                    }
                }
            fft_b<BN, false>(o, v, h, tw);
#pragma unroll
            for (int k1 = 0; k1 < BN; ++k1) {
                const int x = t + 16 * k1;
                if ((unsigned)(sfreq_kk(x, n) - kx0 + n) % (unsigned)n < (unsigned)nbx) gr[64 * k1] = v[k1];
            }
        }
        __syncthreads();
        // P4: band columns, forward along y, series normalisation, band rows stored
        for (int c = hw; c < nbx; c += kKKHW) {
            const int x = freq_index(kx0 + c, n);
            float2 v[BN], o[S][16];
            const int cx = t4_col(x);
            const float2* gc = G + lrow + cx;
#pragma unroll
            for (int j = 0; j < BN; ++j) v[j] = gc[16 * j * n];
            fft_a<BN, false>(v, o, h, tw);
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (t + 16 * s < BN) {
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) {
                        const int y = t + 16 * s + BN * k1;
                        if ((unsigned)(sfreq_kk(y, n) - ky0 + n) % (unsigned)n < (unsigned)nby)
                            G[t4_row(y, n) + cx] = cscale(o[s][k1], inv_n2);
                    }
                }
        }
        __syncthreads();
        float2* out = xdisc + ((size_t)tile * P.n_bf + i) * P.npup;
        for (int p = threadIdx.x; p < P.npup; p += blockDim.x) {
            const int Kx = P.pup_x[p] - kix, Ky = P.pup_y[p] - kiy;
            out[p] = G[t4_index(freq_index(Ky, n), freq_index(Kx, n), n)];
        }
        __syncthreads();
    }
}

using KKRKernel = void (*)(DevPlan, int, const float*, float2*, float2*, const int32_t*);

static KKRKernel kkr_kernel(int BN) {
    switch (BN) {
        case 4: return k_kk_reg<4>;
        case 8: return k_kk_reg<8>;
        case 16: return k_kk_reg<16>;
        case 32: return k_kk_reg<32>;
        default: return nullptr;
    }
}

int configure_kkr(int BN, size_t smem) {
    KKRKernel f = kkr_kernel(BN);
    if (!f) return 0;
    if (smem > 48 * 1024 &&
        raise_smem_limit((const void*)f, smem) != cudaSuccess)
        return 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kKKThreads, smem) != cudaSuccess) return 0;
    return occ;
}

cudaError_t launch_kk_reg(const DevPlan& P, int grid, size_t smem, int n_tiles, const float* I, float2* xdisc,
                          float2* scratch, const int32_t* status, cudaStream_t st) {
    KKRKernel f = kkr_kernel(P.h / 16);
    if (!f) return cudaErrorInvalidValue;
    grid = min(grid, n_tiles * P.n_bf);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    f<<<grid, kKKThreads, smem, st>>>(P, n_tiles, I, xdisc, scratch, status);
    return cudaGetLastError();
}

}  // namespace apic
