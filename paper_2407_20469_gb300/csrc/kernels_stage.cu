// kernels_stage.cu - per-tile stages before the darkfield extension:
// background statistic (Sec. 3.2), Kramers-Kronig recovery (Eq. 4-7),
// aberration solve (Eq. 8-10), pupil-phase table, correction and stitching,
// pupil output.
#include <math.h>

#include "../../include/apic.h"
#include "passes.cuh"
#include "zernike.h"

namespace apic {

// ---------------------------------------------------------------- background
// Per tile: mean over the NA-matching images of var(I)/mean(I)^2; flags
// tiles below the threshold and stacks with negative or non-finite values.
// Each thread sums its own pixels in FP32 (a few hundred values), the block
// combines the partial sums in FP64; the darkfield images are only checked.
__global__ void __launch_bounds__(kThreads) k_background(DevPlan P, int n_tiles, const float* __restrict__ I,
                                                         float* __restrict__ c2, int32_t* __restrict__ status,
                                                         float thresh2, int learned) {
    __shared__ double red[64];
    const int tile = blockIdx.x;
    if (tile >= n_tiles) return;
    const size_t npix = (size_t)P.h * P.w;
    const float* T = I + (size_t)tile * P.n_img * npix;
    double acc = 0;
    int bad = 0, par = 0;
    auto invalid = [](float4 v) {
        return !(v.x >= 0.f && v.x < INFINITY) || !(v.y >= 0.f && v.y < INFINITY) ||
               !(v.z >= 0.f && v.z < INFINITY) || !(v.w >= 0.f && v.w < INFINITY);
    };
    for (int i = 0; i < P.n_img; ++i) {
        const float4* T4 = reinterpret_cast<const float4*>(T + i * npix);
        const int nq = (int)(npix / 4);
        if (i < P.n_bf) {
            float s = 0.f, s2 = 0.f;
#pragma unroll 4
            for (int k = threadIdx.x; k < nq; k += blockDim.x) {
                const float4 v = __ldcs(T4 + k);        // streamed: evict first from L2
                bad |= invalid(v);
                s += (v.x + v.y) + (v.z + v.w);
                s2 += (v.x * v.x + v.y * v.y) + (v.z * v.z + v.w * v.w);
            }
            const double st = block_sum2((double)s, red, par);
            const double st2 = block_sum2((double)s2, red, par);
            const double mean = st / npix;
            const double var = st2 / npix - mean * mean;
            acc += mean > 0 ? var / (mean * mean) : 0.0;
        } else {
#pragma unroll 4
            for (int k = threadIdx.x; k < nq; k += blockDim.x) bad |= invalid(__ldcs(T4 + k));
        }
    }
    const int anybad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        const float v = (float)(acc / P.n_bf);
        if (c2) c2[tile] = v;
        int st = 0;
        if (v < thresh2) st |= learned ? APIC_TILE_LEARNED : APIC_TILE_BACKGROUND;
        if (anybad) st |= APIC_TILE_BADINPUT;
        status[tile] = st;
    }
}

cudaError_t launch_background(const DevPlan& P, int n_tiles, const float* I, float* c2, int32_t* status,
                              float thresh2, cudaStream_t st, int learned) {
    k_background<<<n_tiles, kThreads, 0, st>>>(P, n_tiles, I, c2, status, thresh2, learned);
    return cudaGetLastError();
}

__device__ __forceinline__ bool skip_tile(const int32_t* status, int tile) {
    return status && (status[tile] & (APIC_TILE_BACKGROUND | APIC_TILE_BADINPUT));
}

// ---------------------------------------------------------------- Kramers-Kronig
// One block per (tile, NA-matching image) problem, persistent over problems.
// Scratch: an n x n complex grid per block.
//   P1 rows: log(max(I, 1e-6 mean I)), forward transform along x
//   P2 cols: forward along y, half-plane mask of Eq. 5, inverse along y
//   P3 rows: inverse along x, / n^2, exp (Eq. 6), forward along x
//   P4 cols: forward along y, / n^2 (series coefficients, Eq. 7)
// then the values at K = k_p - k_i for every pupil point k_p are gathered.
__global__ void __launch_bounds__(kThreads) k_kk(DevPlan P, int n_tiles, const float* __restrict__ I,
                                                 float2* __restrict__ xdisc, float2* __restrict__ scratch,
                                                 const int32_t* __restrict__ status) {
    extern __shared__ float4 smem4[];
    float2* sm = reinterpret_cast<float2*>(smem4);
    const int n = P.h, ln = ilog2(n);
    float2* tw = sm + 2 * (kChunk / n) * (n + 1);
    double* red = reinterpret_cast<double*>(tw + n);
    load_twiddles(tw, P.tw_n, n);
    const FFTChunk c = make_chunk(sm, n, tw);
    const int S = c.S, ld = c.ld;
    float2* G = scratch + (size_t)blockIdx.x * n * n;
    const float inv_n2 = 1.0f / (float)(n * n);
    const int nprob = n_tiles * P.n_bf;
    for (int prob = blockIdx.x; prob < nprob; prob += gridDim.x) {
        const int tile = prob / P.n_bf, i = prob - tile * P.n_bf;
        if (skip_tile(status, tile)) continue;
        const float* img = I + ((size_t)tile * P.n_img + i) * n * n;
        const int kix = P.led_x[i], kiy = P.led_y[i];
        double s = 0;
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) s += img[t];
        s = block_sum(s, red);
        const float eps = (float)(1e-6 * s / ((double)n * n));
        // P1
        for (int r0 = 0; r0 < n; r0 += S) {
            for (int t = threadIdx.x; t < (S << ln); t += blockDim.x) {
                const int q = t >> ln, x = t & (n - 1);
                c.a[q * ld + x] = make_float2(logf(fmaxf(img[(size_t)(r0 + q) * n + x], eps)), 0.f);
            }
            const float2* R = fft_chunk<false>(c);
            for (int t = threadIdx.x; t < (S << ln); t += blockDim.x) {
                const int q = t >> ln, x = t & (n - 1);
                G[(size_t)(r0 + q) * n + x] = R[q * ld + x];
            }
            __syncthreads();
        }
        // P2
        const long long hh = (long long)P.h * P.h, ww = (long long)P.w * P.w;
        for (int c0 = 0; c0 < n; c0 += S) {
            for (int t = threadIdx.x; t < S * n; t += blockDim.x) {
                const int y = t / S, q = t - y * S;
                c.a[q * ld + y] = G[(size_t)y * n + c0 + q];
            }
            float2* R = fft_chunk<false>(c);
            for (int t = threadIdx.x; t < S * n; t += blockDim.x) {
                const int y = t / S, q = t - y * S;
                const long long dot = (long long)signed_freq(c0 + q, n) * kix * hh + (long long)signed_freq(y, n) * kiy * ww;
                const float f = dot < 0 ? 1.f : (dot == 0 ? 0.5f : 0.f);
                R[q * ld + y] = cscale(R[q * ld + y], f);
            }
            FFTChunk c2 = c;
            c2.a = R;
            c2.b = (R == c.a) ? c.b : c.a;
            const float2* R2 = fft_chunk<true>(c2);
            for (int t = threadIdx.x; t < S * n; t += blockDim.x) {
                const int y = t / S, q = t - y * S;
                G[(size_t)y * n + c0 + q] = R2[q * ld + y];
            }
            __syncthreads();
        }
        // P3
        for (int r0 = 0; r0 < n; r0 += S) {
            for (int t = threadIdx.x; t < (S << ln); t += blockDim.x) {
                const int q = t >> ln, x = t & (n - 1);
                c.a[q * ld + x] = G[(size_t)(r0 + q) * n + x];
            }
            float2* R = fft_chunk<true>(c);
            for (int t = threadIdx.x; t < (S << ln); t += blockDim.x) {
                const int q = t >> ln, x = t & (n - 1);
                const float2 z = cscale(R[q * ld + x], inv_n2);
                float sn, cs;
                sincosf(z.y, &sn, &cs);
                const float e = expf(z.x);
                R[q * ld + x] = make_float2(e * cs, e * sn);
            }
            FFTChunk c2 = c;
            c2.a = R;
            c2.b = (R == c.a) ? c.b : c.a;
            const float2* R2 = fft_chunk<false>(c2);
            for (int t = threadIdx.x; t < (S << ln); t += blockDim.x) {
                const int q = t >> ln, x = t & (n - 1);
                G[(size_t)(r0 + q) * n + x] = R2[q * ld + x];
            }
            __syncthreads();
        }
        // P4
        for (int c0 = 0; c0 < n; c0 += S) {
            for (int t = threadIdx.x; t < S * n; t += blockDim.x) {
                const int y = t / S, q = t - y * S;
                c.a[q * ld + y] = G[(size_t)y * n + c0 + q];
            }
            const float2* R = fft_chunk<false>(c);
            for (int t = threadIdx.x; t < S * n; t += blockDim.x) {
                const int y = t / S, q = t - y * S;
                G[(size_t)y * n + c0 + q] = cscale(R[q * ld + y], inv_n2);
            }
            __syncthreads();
        }
        float2* out = xdisc + ((size_t)tile * P.n_bf + i) * P.npup;
        for (int p = threadIdx.x; p < P.npup; p += blockDim.x) {
            const int Kx = P.pup_x[p] - kix, Ky = P.pup_y[p] - kiy;
            out[p] = G[(size_t)freq_index(Ky, n) * n + freq_index(Kx, n)];
        }
        __syncthreads();
    }
}

cudaError_t launch_kk(const DevPlan& P, const Launch& L, int n_tiles, const float* I, float2* xdisc,
                      float2* scratch, const int32_t* status, cudaStream_t st) {
    const int grid = min(L.grid_kk, n_tiles * P.n_bf);
    k_kk<<<grid, kThreads, L.smem_kk, st>>>(P, n_tiles, I, xdisc, scratch, status);
    return cudaGetLastError();
}

cudaError_t launch_kk_grid(const DevPlan& P, int grid, size_t smem, int n_tiles, const float* I, float2* xdisc,
                           float2* scratch, const int32_t* status, cudaStream_t st) {
    grid = min(grid, n_tiles * P.n_bf);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    k_kk<<<grid, kThreads, smem, st>>>(P, n_tiles, I, xdisc, scratch, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- aberration
// One block per tile (persistent). beta(r) = arg(X_i X_l^*) on every overlap
// row (Eq. 9). Stage 1 fits the wrapped differences of neighbouring rows,
// stage 2 runs `passes` refinements on the rows of Eq. 10. Products are
// accumulated per thread in FP32, summed across the block in FP64, and the
// 12 x 12 normal equations are solved in FP64 with the plan's Cholesky factors.
__device__ void reduce12(float* g, double* red, double* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int z = 0; z < 12; ++z) {
        double v = g[z];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp * 12 + z] = v;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        double t = 0;
        for (int w = 0; w < nw; ++w) t += red[w * 12 + threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

__device__ void chol_solve12(const double* L, const double* b, double* x) {
    double y[12];
    for (int i = 0; i < 12; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * 12 + k] * y[k];
        y[i] = s / L[i * 12 + i];
    }
    for (int i = 11; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 12; ++k) s -= L[k * 12 + i] * x[k];
        x[i] = s / L[i * 12 + i];
    }
}

// Refinement passes c <- c + LS(wrap(beta - D c)) from the coefficients in
// cc / cf (shared); returns the sum of squared wrapped residuals of the rows
// at the final coefficients (every thread gets it).
__device__ double value_passes(const DevPlan& P, const float* beta, int passes, double* cc, float* cf, double* dc,
                               double* rhs, double* red) {
    float g[12];
    for (int pass = 0; pass < passes; ++pass) {
        for (int z = 0; z < 12; ++z) g[z] = 0.f;
        for (int r = threadIdx.x; r < P.nrows; r += blockDim.x) {
            const float* A = P.row_A + (size_t)r * 12;
            float pred = 0.f;
            for (int z = 0; z < 12; ++z) pred += A[z] * cf[z];
            const float e = wrap_pi(beta[r] - pred);
            for (int z = 0; z < 12; ++z) g[z] += A[z] * e;
        }
        reduce12(g, red, rhs);
        if (threadIdx.x == 0) {
            chol_solve12(P.Lval, rhs, dc);
            for (int z = 0; z < 12; ++z) {
                cc[z] += dc[z];
                cf[z] = (float)cc[z];
            }
        }
        __syncthreads();
    }
    double res = 0;
    for (int r = threadIdx.x; r < P.nrows; r += blockDim.x) {
        const float* A = P.row_A + (size_t)r * 12;
        float pred = 0.f;
        for (int z = 0; z < 12; ++z) pred += A[z] * cf[z];
        const float e = wrap_pi(beta[r] - pred);
        res += (double)(e * e);
    }
    return block_sum(res, red);
}

// c0 [tiles][15] (may be NULL): learned coefficients. Tiles marked
// APIC_TILE_LEARNED take c0 as their result. With `warm`, every solved tile
// also runs the refinement passes from c0 and keeps whichever of the two
// solutions leaves the smaller wrapped residual (then sets APIC_TILE_WARM).
__global__ void __launch_bounds__(kThreads) k_aberration(DevPlan P, int n_tiles, const float2* __restrict__ xdisc,
                                                         float* __restrict__ zern, float* __restrict__ beta_scratch,
                                                         int passes, int32_t* __restrict__ status,
                                                         const float* __restrict__ c0, int warm) {
    __shared__ double red[16 * 12];
    __shared__ double rhs[12], cc[12], dc[12], cbest[12];
    __shared__ float cf[12];
    float* beta = beta_scratch + (size_t)blockIdx.x * P.nrows;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (skip_tile(status, tile)) {
            if (threadIdx.x < APIC_N_ZERNIKE) zern[(size_t)tile * APIC_N_ZERNIKE + threadIdx.x] = 0.f;
            continue;
        }
        if (c0 && status && (status[tile] & APIC_TILE_LEARNED)) {
            if (threadIdx.x < APIC_N_ZERNIKE)
                zern[(size_t)tile * APIC_N_ZERNIKE + threadIdx.x] =
                    threadIdx.x < 3 ? 0.f : c0[(size_t)tile * APIC_N_ZERNIKE + threadIdx.x];
            continue;
        }
        const float2* X = xdisc + (size_t)tile * P.n_bf * P.npup;
        for (int r = threadIdx.x; r < P.nrows; r += blockDim.x) {
            const int il = P.row_il[r];
            const float2 a = X[(size_t)(il & 0xffff) * P.npup + P.row_pi[r]];
            const float2 b = X[(size_t)(il >> 16) * P.npup + P.row_pl[r]];
            const float2 z = cmulc(a, b);
            beta[r] = atan2f(z.y, z.x);
        }
        __syncthreads();
        float g[12];
        for (int z = 0; z < 12; ++z) g[z] = 0.f;
        for (int r = threadIdx.x; r < P.nrows; r += blockDim.x) {
            const float* A = P.row_A + (size_t)r * 12;
            const float br = beta[r];
            const int nb[2] = {P.row_nx[r], P.row_ny[r]};
            for (int d = 0; d < 2; ++d) {
                if (nb[d] < 0) continue;
                const float* A2 = P.row_A + (size_t)nb[d] * 12;
                const float e = wrap_pi(beta[nb[d]] - br);
                for (int z = 0; z < 12; ++z) g[z] += (A2[z] - A[z]) * e;
            }
        }
        reduce12(g, red, rhs);
        if (threadIdx.x == 0) {
            chol_solve12(P.Lgrad, rhs, cc);
            for (int z = 0; z < 12; ++z) cf[z] = (float)cc[z];
        }
        __syncthreads();
        bool won = false;
        if (c0 && warm) {
            const double res = value_passes(P, beta, passes, cc, cf, dc, rhs, red);
            if (threadIdx.x < 12) {
                cbest[threadIdx.x] = cc[threadIdx.x];
                cc[threadIdx.x] = c0[(size_t)tile * APIC_N_ZERNIKE + 3 + threadIdx.x];
                cf[threadIdx.x] = (float)cc[threadIdx.x];
            }
            __syncthreads();
            const double res_w = value_passes(P, beta, passes, cc, cf, dc, rhs, red);
            won = res_w < res;
            if (!won && threadIdx.x < 12) cc[threadIdx.x] = cbest[threadIdx.x];
            __syncthreads();
        } else {
            value_passes(P, beta, passes, cc, cf, dc, rhs, red);
        }
        if (threadIdx.x < APIC_N_ZERNIKE)
            zern[(size_t)tile * APIC_N_ZERNIKE + threadIdx.x] = threadIdx.x < 3 ? 0.f : (float)cc[threadIdx.x - 3];
        if (won && status && threadIdx.x == 0) status[tile] |= APIC_TILE_WARM;
        __syncthreads();
    }
}

cudaError_t launch_aberration(const DevPlan& P, const Launch& L, int n_tiles, const float2* xdisc, float* zern,
                              float* beta_scratch, int passes, int32_t* status, cudaStream_t st, const float* c0,
                              int warm) {
    const int grid = min(L.grid_ab, n_tiles);
    k_aberration<<<grid, kThreads, 0, st>>>(P, n_tiles, xdisc, zern, beta_scratch, passes, status, c0, warm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- phase table
// phi[tile][p] = sum_j c_j Z_j(k_p / R) at every pupil point.
__global__ void k_phase(DevPlan P, int n_tiles, const float* __restrict__ zern, float* __restrict__ phi) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n_tiles * P.npup) return;
    const int tile = (int)(idx / P.npup), p = (int)(idx - (size_t)tile * P.npup);
    float z[12];
    zernike_4_15<float>((float)P.pup_x[p] / P.Rx, (float)P.pup_y[p] / P.Ry, z);
    const float* c = zern + (size_t)tile * APIC_N_ZERNIKE + 3;
    float v = 0.f;
    for (int j = 0; j < 12; ++j) v += c[j] * z[j];
    phi[idx] = v;
}

cudaError_t launch_phase(const DevPlan& P, int n_tiles, const float* zern, float* phi, cudaStream_t st) {
    const size_t total = (size_t)n_tiles * P.npup;
    k_phase<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, n_tiles, zern, phi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- stitch
// Corrected spectrum X_i(K) exp(-j[phi(K + k_i) - phi(k_i)]) averaged over the
// discs covering each aperture point; zero where only darkfield reaches.
__global__ void k_stitch(DevPlan P, int n_tiles, const float2* __restrict__ xdisc, const float* __restrict__ phi,
                         float2* __restrict__ spec, const int32_t* __restrict__ status) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n_tiles * P.nap) return;
    const int tile = (int)(idx / P.nap), a = (int)(idx - (size_t)tile * P.nap);
    if (skip_tile(status, tile)) {
        spec[idx] = make_float2(0.f, 0.f);
        return;
    }
    const float* ph = phi + (size_t)tile * P.npup;
    const float2* X = xdisc + (size_t)tile * P.n_bf * P.npup;
    float2 acc = make_float2(0.f, 0.f);
    const int e0 = P.st_ptr[a], e1 = P.st_ptr[a + 1];
    for (int e = e0; e < e1; ++e) {
        const int i = P.st_img[e], p = P.st_pup[e];
        float sn, cs;
        sincosf(ph[p] - ph[P.led_pup[i]], &sn, &cs);
        acc = cadd(acc, cmul(X[(size_t)i * P.npup + p], make_float2(cs, -sn)));
    }
    spec[idx] = e1 > e0 ? cscale(acc, 1.f / (float)(e1 - e0)) : make_float2(0.f, 0.f);
}

cudaError_t launch_stitch(const DevPlan& P, int n_tiles, const float2* xdisc, const float* phi, float2* spec,
                          const int32_t* status, cudaStream_t st) {
    const size_t total = (size_t)n_tiles * P.nap;
    k_stitch<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, n_tiles, xdisc, phi, spec, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- pupil
__global__ void k_pupil(DevPlan P, int n_tiles, const float* __restrict__ phi, float2* __restrict__ pupil,
                        const int32_t* __restrict__ status) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t npix = (size_t)P.h * P.w;
    if (idx >= (size_t)n_tiles * npix) return;
    const int tile = (int)(idx / npix);
    const int r = (int)(idx - (size_t)tile * npix);
    const int ky = signed_freq(r / P.w, P.h), kx = signed_freq(r % P.w, P.w);
    float2 v = make_float2(0.f, 0.f);
    if (!skip_tile(status, tile) && kx >= -P.pup_ax && kx <= P.pup_ax && ky >= -P.pup_ay && ky <= P.pup_ay) {
        const int p = P.pup_lut[(ky + P.pup_ay) * (2 * P.pup_ax + 1) + kx + P.pup_ax];
        if (p >= 0) {
            float sn, cs;
            sincosf(phi[(size_t)tile * P.npup + p], &sn, &cs);
            v = make_float2(cs, sn);
        }
    }
    pupil[idx] = v;
}

cudaError_t launch_pupil(const DevPlan& P, int n_tiles, const float* phi, float2* pupil, const int32_t* status,
                         cudaStream_t st) {
    const size_t total = (size_t)n_tiles * P.h * P.w;
    k_pupil<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, n_tiles, phi, pupil, status);
    return cudaGetLastError();
}

}  // namespace apic

namespace apic {
__global__ void k_darkfield(DevPlan, int, const float*, const float*, float2*, char*, size_t, int, float, int32_t*,
                            unsigned long long*);
__global__ void k_synthesize(DevPlan, int, const float2*, float2*, const int32_t*);
__global__ void k_sim_images(DevPlan, int, const float2*, const float*, float, unsigned long long, float*, float2*);
__global__ void k_sim_object(DevPlan, int, const float2*, float2*);

int configure_kernel(int which, size_t smem) {
    const void* f = nullptr;
    switch (which) {
        case 0: f = (const void*)k_kk; break;
        case 1: f = (const void*)k_aberration; break;
        case 2: f = (const void*)k_darkfield; break;
        case 3: f = (const void*)k_synthesize; break;
        case 4: f = (const void*)k_sim_images; break;
        case 5: f = (const void*)k_sim_object; break;
        default: return 0;
    }
    if (smem > 48 * 1024 && raise_smem_limit(f, smem) != cudaSuccess)
        return 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kThreads, smem) != cudaSuccess) return 0;
    return occ;
}
}  // namespace apic
