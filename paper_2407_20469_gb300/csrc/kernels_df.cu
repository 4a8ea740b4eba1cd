// kernels_df.cu - darkfield spectrum extension (WSI-APIC Eq. 11-13).
//
// For each darkfield image j (plan order), in the pupil frame c = K + k_j:
//   U: unknown disc points, P: known disc points, Q: lags of Eq. 13.
//   b(k)   = F(I_j)(k) - (P*P)(k),            k in Q
//   (C u)(k) = sum_{q in U} u(q) conj P(q - k)  = series coefficient at k of
//              u(x) conj p(x), with u, p the fields synthesised from U and P.
//   (C^H r)(q) = sum_{k in Q} r(k) P(q - k)    = series coefficient at q of
//              v(x) p(x), v synthesised from r.
// Both products are evaluated on an m x m grid with m > 4 max|c| (alias free)
// by band-limited row passes and full column passes. The least-squares problem
// min ||C u - b|| is solved by CGLS: transforms in FP32, inner products and
// the step lengths in FP64, the solution accumulated in FP64. The object
// spectrum gains O(K) = u(c) exp(-j phi(c)) on U.
//
// One block per tile (persistent); the darkfield images of a tile are
// sequential because each one's known set includes the previous unknowns.
#include <math.h>

#include "../../include/apic.h"
#include "passes.cuh"

namespace apic {

size_t df_scratch_bytes(const DevPlan& P) {
    const size_t g = (size_t)max(P.h * P.w, P.m * P.m);
    size_t b = g * sizeof(float2) + (size_t)P.m * P.m * sizeof(float2);
    b += (size_t)P.max_N * sizeof(double2) + 2 * (size_t)P.max_N * sizeof(float2) + 2 * (size_t)P.max_M * sizeof(float2);
    return (b + 255) & ~(size_t)255;
}

__global__ void __launch_bounds__(kThreads) k_darkfield(DevPlan P, int n_tiles, const float* __restrict__ I,
                                                        const float* __restrict__ phi, float2* __restrict__ spec,
                                                        char* __restrict__ scratch, size_t per_block, int iters,
                                                        float tol, int32_t* __restrict__ status,
                                                        unsigned long long* __restrict__ counters) {
    extern __shared__ float4 smem4[];
    float2* sm = reinterpret_cast<float2*>(smem4);
    const int n = P.h, m = P.m;
    const int bufN = max(2 * (kChunk / n) * (n + 1), 2 * (kChunk / m) * (m + 1));
    float2* tw_n = sm + bufN;
    float2* tw_m = tw_n + n;
    double* red = reinterpret_cast<double*>(tw_m + m);
    load_twiddles(tw_n, P.tw_n, n);
    load_twiddles(tw_m, P.tw_m, m);
    const FFTChunk cn = make_chunk(sm, n, tw_n);
    const FFTChunk cm = make_chunk(sm, m, tw_m);

    char* base = scratch + (size_t)blockIdx.x * per_block;
    float2* G = reinterpret_cast<float2*>(base);
    float2* PF = G + max(n * n, m * m);
    double2* xv = reinterpret_cast<double2*>(PF + (size_t)m * m);
    float2* dv = reinterpret_cast<float2*>(xv + P.max_N);
    float2* sv = dv + P.max_N;
    float2* rv = sv + P.max_N;
    float2* qv = rv + P.max_M;

    const float inv_n2 = 1.f / (float)(n * n), inv_m2 = 1.f / (float)(m * m);
    const int ldm = cm.ld, Sm = cm.S, lm = cm.logN;

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (status && (status[tile] & (APIC_TILE_BACKGROUND | APIC_TILE_BADINPUT))) continue;
        const float* ph = phi + (size_t)tile * P.npup;
        float2* sp = spec + (size_t)tile * P.nap;
        bool notconv = false;
        for (int di = 0; di < P.n_used; ++di) {
            const DevDF D = P.df[di];
            const int *Ux = P.dU_x + D.u_off, *Uy = P.dU_y + D.u_off;
            const int *Upup = P.dU_pup + D.u_off, *Uap = P.dU_ap + D.u_off;
            const int *Px = P.dP_x + D.p_off, *Py = P.dP_y + D.p_off;
            const int *Ppup = P.dP_pup + D.p_off, *Pap = P.dP_ap + D.p_off;
            const int *Qx = P.dQ_x + D.q_off, *Qy = P.dQ_y + D.q_off;
            const int *urp = P.d_rowptr + D.urp, *qrp = P.d_rowptr + D.qrp, *prp = P.d_rowptr + D.prp;
            const float* img = I + ((size_t)tile * P.n_img + D.led) * n * n;
            const int N = D.N, M = D.M;

            // ---- b = F(I_j) on Q: columns of the image forward along y, then rows
            {
                const int S = cn.S, ld = cn.ld, nbq = D.qy1 - D.qy0 + 1;
                for (int c0 = 0; c0 < n; c0 += S) {
                    if (D.tr) {   // the transposed image (solve frame with x <-> y)
                        for (int t = threadIdx.x; t < S * n; t += blockDim.x) {
                            const int q = t / n, y = t - q * n;
                            cn.a[q * ld + y] = make_float2(img[(size_t)(c0 + q) * n + y], 0.f);
                        }
                    } else {
                        for (int t = threadIdx.x; t < S * n; t += blockDim.x) {
                            const int y = t / S, q = t - y * S;
                            cn.a[q * ld + y] = make_float2(img[(size_t)y * n + c0 + q], 0.f);
                        }
                    }
                    const float2* R = fft_chunk<false>(cn);
                    for (int t = threadIdx.x; t < nbq * S; t += blockDim.x) {
                        const int b = t / S, q = t - b * S;
                        const int y = freq_index(D.qy0 + b, n);
                        G[(size_t)y * n + c0 + q] = R[q * ld + y];
                    }
                    __syncthreads();
                }
                rows_to_points(cn, G, n, D.qy0, D.qy1, qrp, Qx, Qy,
                               [&](int e, float2 v) { rv[e] = cscale(v, inv_n2); });
            }
            // ---- known field p(x) from P (kept in PF), and b -= (P*P) on Q
            rows_from_points<true>(cm, G, m, D.py0, D.py1, prp, Px, Py, [&](int e) {
                float sn, cs;
                sincosf(ph[Ppup[e]], &sn, &cs);
                return cmul(sp[Pap[e]], make_float2(cs, sn));
            });
            cols_inv_mid_fwd(cm, G, m, D.py0, D.py1, D.qy0, D.qy1, [&](float2* R, int c0) {
                for (int t = threadIdx.x; t < (Sm << lm); t += blockDim.x) {
                    const int y = t / Sm, q = t - y * Sm;
                    const float2 v = R[q * ldm + y];
                    PF[(size_t)y * m + c0 + q] = v;
                    R[q * ldm + y] = make_float2(cabs2(v), 0.f);
                }
            });
            rows_to_points(cm, G, m, D.qy0, D.qy1, qrp, Qx, Qy,
                           [&](int e, float2 v) { rv[e] = csub(rv[e], cscale(v, inv_m2)); });
            __syncthreads();

            // ---- the two correlation operators
            auto apply_CH = [&]() -> double {   // sv = C^H rv, returns ||sv||^2
                rows_from_points<true>(cm, G, m, D.qy0, D.qy1, qrp, Qx, Qy, [&](int e) { return rv[e]; });
                cols_inv_mid_fwd(cm, G, m, D.qy0, D.qy1, D.uy0, D.uy1, [&](float2* R, int c0) {
                    for (int t = threadIdx.x; t < (Sm << lm); t += blockDim.x) {
                        const int y = t / Sm, q = t - y * Sm;
                        R[q * ldm + y] = cscale(cmul(R[q * ldm + y], PF[(size_t)y * m + c0 + q]), inv_m2);
                    }
                });
                double acc = 0;
                rows_to_points(cm, G, m, D.uy0, D.uy1, urp, Ux, Uy, [&](int e, float2 v) {
                    sv[e] = v;
                    acc += (double)v.x * v.x + (double)v.y * v.y;
                });
                return block_sum(acc, red);
            };
            auto apply_C = [&]() -> double {    // qv = C dv, returns ||qv||^2
                rows_from_points<true>(cm, G, m, D.uy0, D.uy1, urp, Ux, Uy, [&](int e) { return dv[e]; });
                cols_inv_mid_fwd(cm, G, m, D.uy0, D.uy1, D.qy0, D.qy1, [&](float2* R, int c0) {
                    for (int t = threadIdx.x; t < (Sm << lm); t += blockDim.x) {
                        const int y = t / Sm, q = t - y * Sm;
                        R[q * ldm + y] = cscale(cmulc(R[q * ldm + y], PF[(size_t)y * m + c0 + q]), inv_m2);
                    }
                });
                double acc = 0;
                rows_to_points(cm, G, m, D.qy0, D.qy1, qrp, Qx, Qy, [&](int e, float2 v) {
                    qv[e] = v;
                    acc += (double)v.x * v.x + (double)v.y * v.y;
                });
                return block_sum(acc, red);
            };

            // ---- CGLS
            for (int e = threadIdx.x; e < N; e += blockDim.x) xv[e] = make_double2(0.0, 0.0);
            const double gamma0 = apply_CH();
            for (int e = threadIdx.x; e < N; e += blockDim.x) dv[e] = sv[e];
            __syncthreads();
            double gamma = gamma0;
            bool conv = !(gamma0 > 1e-300);
            const double stop = (double)tol * (double)tol * gamma0;
            int it = 0;
            for (; it < iters && !conv; ++it) {
                const double delta = apply_C();
                if (!(delta > 0)) break;
                const double alpha = gamma / delta;
                for (int e = threadIdx.x; e < N; e += blockDim.x) {
                    const float2 d = dv[e];
                    double2 x = xv[e];
                    x.x += alpha * d.x;
                    x.y += alpha * d.y;
                    xv[e] = x;
                }
                const float af = (float)alpha;
                for (int e = threadIdx.x; e < M; e += blockDim.x) rv[e] = csub(rv[e], cscale(qv[e], af));
                __syncthreads();
                const double gnew = apply_CH();
                const float bf = (float)(gnew / gamma);
                gamma = gnew;
                for (int e = threadIdx.x; e < N; e += blockDim.x) dv[e] = cadd(sv[e], cscale(dv[e], bf));
                __syncthreads();
                conv = gnew <= stop;
            }
            if (!conv) notconv = true;
            if (threadIdx.x == 0 && counters) {
                atomicAdd(counters + 1, (unsigned long long)it);
                atomicAdd(counters + 2, 1ull);
                if (di < kCountedImages) atomicAdd(counters + 4 + di, (unsigned long long)it);
            }
            // ---- O(K) = u(c) exp(-j phi(c)) on U
            for (int e = threadIdx.x; e < N; e += blockDim.x) {
                float sn, cs;
                sincosf(ph[Upup[e]], &sn, &cs);
                const double2 x = xv[e];
                sp[Uap[e]] = cmul(make_float2((float)x.x, (float)x.y), make_float2(cs, -sn));
            }
            __syncthreads();
        }
        if (threadIdx.x == 0 && notconv && status) atomicOr(status + tile, APIC_TILE_NOTCONV);
    }
}

cudaError_t launch_darkfield(const DevPlan& P, const Launch& L, int n_tiles, const float* I, const float* phi,
                             float2* spec, void* scratch, size_t scratch_per_block, int iters, float tol,
                             int32_t* status, unsigned long long* counters, cudaStream_t st) {
    const int grid = min(L.grid_df, n_tiles);
    k_darkfield<<<grid, kThreads, L.smem_df, st>>>(P, n_tiles, I, phi, spec, (char*)scratch, scratch_per_block,
                                                   iters, tol, status, counters);
    return cudaGetLastError();
}

}  // namespace apic
