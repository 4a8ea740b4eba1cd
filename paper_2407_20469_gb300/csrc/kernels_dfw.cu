// kernels_dfw.cu - darkfield spectrum extension (WSI-APIC Eq. 11-13) for 512-pixel
// tiles, with the wide register FFTs (16 B points, 16 < B <= 32, two step-B rows
// per lane).
//
// The method is the one of kernels_dfr.cu (CG on the normal equations of Eq. 13,
// five passes per iteration over a band-row grid; see there), at the sizes of a
// 512 x 512 tile (pupil radius ~85 grid points, up to ~2.8 k unknowns and ~36 k
// equations per image):
//  * the right-hand side b = F(I_j) - P * P on Q is formed on the camera grid,
//    n = 512 = 16 x 32, as the spectrum of I_j - |p|^2 with p the known field's
//    inverse transform (exact: the lags of P * P reach 2 R < n / 2);
//  * each image's CG runs on its own (row, column) grid chosen with the plan,
//    rows of 288 or 320 points and columns of 192, 256, 288 or 320 points, the
//    smallest on which both correlations are free of aliasing;
//  * the band grids GU, GQ, the column-major known field p and b on Q live in the
//    block's global scratch (L2 / HBM): a 512-pixel tile's GU alone (up to 94 rows
//    of 320 points) exceeds what shared memory can hold beside the transform
//    areas. The band grids are stored in 4 x 4 tiles (t4_index), so that the column
//    passes' loads and stores use whole sectors and few cache lines, like the rows
//    passes'. Shared memory holds the half-warp transform areas and the CG vectors;
//    the setup transforms (512-point areas, the column stage) alias both, since no
//    CG vector is live while an image is being set up.
// A tile is solved by a cluster of K blocks of 512 threads (persistent over tiles;
// images of a tile in order): every pass splits its rows or columns over the K x 32
// half-warps of the cluster, each block owning a fixed share (and with it the CG
// vector entries of its U rows); passes end at cluster barriers and inner products
// are summed across the blocks through distributed shared memory, in rank order, so
// every block takes the same steps. With K blocks per tile only 1/K as many tiles are
// in flight, so their band grids stay in L2 instead of going to HBM. Data another
// block wrote is read with L2-only loads (no stale L1 lines).
// Transforms, vectors and per-thread / per-warp partial sums FP32; the sums across
// warps and blocks and the CG step lengths FP64.
#include <math.h>

#include <algorithm>

#include "../../include/apic.h"
#include "internal.cuh"
#include "regfft.cuh"
#include "t4grid.cuh"

namespace apic {

namespace {

#ifndef APIC_DFW_THREADS
#define APIC_DFW_THREADS 512
#endif
constexpr int kWThreads = APIC_DFW_THREADS;
constexpr int kWHW = kWThreads / 16;       // half-warps per block
constexpr int kWStageLd = 33;              // column stage: 32 columns + 1 pad
constexpr int kWBN = 32;                   // camera grid 16 x 32 = 512
constexpr int kWMaxB = 20;                 // longest CG grid: 16 x 20 = 320 points
constexpr int kWQWords = 16;               // Q membership words per band row (two 16-bit masks each)

__device__ __forceinline__ int sfreqw(int i, int n) { return i < n / 2 ? i : i - n; }

// Half-warp of a cluster: t lane, hw index in the block, gh index in the cluster
// (rank x 32 + hw), ghs half-warps in the cluster.
struct HWw {
    int t, hw, gh, ghs;
    unsigned mask;
    float2* hs;
    __device__ HalfWarp h() const { return HalfWarp{t, mask, hs}; }
};

__device__ __forceinline__ unsigned cta_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Barrier of all threads of the K blocks of a tile (release / acquire at cluster
// scope); a block barrier when K = 1.
template <int K>
__device__ __forceinline__ void tile_sync() {
    if constexpr (K == 1) {
        __syncthreads();
    } else {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
}

// Load of scratch data that another block of the cluster may have written: from L2.
template <int K>
__device__ __forceinline__ float2 ldx(const float2* p) {
    if constexpr (K == 1)
        return *p;
    else
        return __ldcg(p);
}

// Sum over the tile's K blocks of FP32 per-thread values: FP32 within warps, FP64
// across the block's warps (warp 0) and across the blocks (each block's total stored
// into slot `rank` of every block's area through distributed shared memory, then
// summed in rank order, so all blocks hold the same value). red: 96 doubles;
// `parity` alternates so that a slot is never rewritten while a block still reads it.
template <int K>
__device__ __forceinline__ double tile_sum(float v, double* red, int& parity) {
    if constexpr (K == 1) {
        return block_sum2f(v, red, parity);
    } else {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
        double* r = red + parity * 32;
        double* slots = red + 64 + parity * 16;
        if (lane == 0) r[warp] = (double)v;
        __syncthreads();
        if (warp == 0) {
            double t = lane < nw ? r[lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane < K) {          // lane q stores this block's total into block q's slot
                const unsigned a = (unsigned)__cvta_generic_to_shared(slots + cta_rank());
                unsigned ra;
                asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"((unsigned)lane));
                asm volatile("st.shared::cluster.f64 [%0], %1;" :: "r"(ra), "d"(t) : "memory");
            }
        }
        tile_sync<K>();
        double total = 0.0;
#pragma unroll
        for (int q = 0; q < K; ++q) total += slots[q];
        parity ^= 1;
        return total;
    }
}

// ---- per-point functors (as in the 256-pixel kernel)
template <int K>
struct WValKnown {      // P(c) = O_known(K) exp(j phi(c)) (the spectrum: written by any block of the tile)
    const float2* sp;
    const float* ph;
    const int* ap;
    const int* pup;
    __device__ float2 operator()(int e) const {
        float sn, cs;
        sincosf(ph[pup[e]], &sn, &cs);
        return cmul(ldx<K>(sp + ap[e]), make_float2(cs, sn));
    }
};
struct WValNextDir {    // d = s + beta d (stored back)
    const float2* sv;
    float2* dv;
    float beta;
    __device__ float2 operator()(int e) const {
        const float2 d = cadd(sv[e], cscale(dv[e], beta));
        dv[e] = d;
        return d;
    }
};
struct WOutStart {      // s = d = C^H b, x = 0; returns |s|^2
    float2* sv;
    float2* dv;
    float2* xv;
    __device__ float operator()(int e, float2 v) const {
        sv[e] = v;
        dv[e] = v;
        xv[e] = make_float2(0.f, 0.f);
        return v.x * v.x + v.y * v.y;
    }
};
struct WValB {          // b on Q
    const float2* bq;
    __device__ float2 operator()(int e) const { return bq[e]; }
};
struct WOutDot {        // w = C^H C d; returns Re <d, w>
    float2* wv;
    const float2* dv;
    __device__ float operator()(int e, float2 v) const {
        wv[e] = v;
        const float2 d = dv[e];
        return d.x * v.x + d.y * v.y;
    }
};

// ---- per-column operations on a column of 16 B points: slot s of lane t holds
// o[s][k1] = the value at y = (t + 16 s) + B k1 (valid where t + 16 s < B)
template <int B>
struct WMidStoreField {     // column-major p s W^(shift k) (16 B values per column; wt: W_16B^j)
    float2* PF;
    float scale;
    const float2* wt;
    int shift;
    static constexpr bool kOut = false;
    static constexpr bool kPre = false;
    __device__ void operator()(float2 (&o)[Slots<B>::value][16], int x, int t) const {
        constexpr int m = 16 * B;
        float2* col = PF + (size_t)x * m;
#pragma unroll
        for (int s = 0; s < Slots<B>::value; ++s)
            if (t + 16 * s < B) {
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) {
                    const int k = t + 16 * s + B * k1;
                    col[k] = cscale(cmul(o[s][k1], wt[(shift * k) % m]), scale);
                }
            }
    }
};
template <int B, bool CONJ>
struct WMidTimesField {     // o *= p s or conj(p s), from the column-major copy
    const float2* PF;
    static constexpr bool kOut = true;
    // 256-point columns: the column's 16 values of this lane are loaded before the
    // forward transform (pre), so that their latency overlaps it (measured on the whole
    // step, same box: 1618 Mpx/s against 1567 with the 192-point columns included;
    // the two-slot columns have no registers for it)
    static constexpr bool kPre = B == 16;
    struct Pre {
        float2 v[16];
    };
    __device__ void load(Pre& p, int x, int t) const {
        const float2* col = PF + (size_t)x * (16 * B) + t;
        if (t < B) {
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) p.v[k1] = col[B * k1];
        }
    }
    __device__ void apply(float2 (&o)[Slots<B>::value][16], const Pre& p) const {
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) o[0][k1] = CONJ ? cmulc(o[0][k1], p.v[k1]) : cmul(o[0][k1], p.v[k1]);
    }
    __device__ void operator()(float2 (&o)[Slots<B>::value][16], int x, int t) const {
        const float2* col = PF + (size_t)x * (16 * B);
#pragma unroll
        for (int s = 0; s < Slots<B>::value; ++s)
            if (t + 16 * s < B) {
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) {
                    const float2 pf = col[t + 16 * s + B * k1];
                    o[s][k1] = CONJ ? cmulc(o[s][k1], pf) : cmul(o[s][k1], pf);
                }
            }
    }
};

// ---- passes (each a separate function so registers are allocated per pass)

// rows of a band: scatter val(e) at x = px[e], inverse transform along x, store the
// rows of the tiled grid G (ld columns).
template <int B, class Val>
__device__ __noinline__ void wpass_rows_in(HWw w, const float2* tw, float2* G, int ld, int nrows, const int* rp,
                                           const int* px, Val val) {
    constexpr int m = 16 * B, S = Slots<B>::value;
    const HalfWarp h = w.h();
    const T4Lane L(w.t);
    for (int b = w.gh; b < nrows; b += w.ghs) {
#pragma unroll
        for (int j = 0; j < B; ++j) w.hs[w.t + 16 * j] = make_float2(0.f, 0.f);
        __syncwarp(w.mask);
        for (int e = rp[b] + w.t; e < rp[b + 1]; e += 16) w.hs[freq_index(px[e], m)] = val(e);
        __syncwarp(w.mask);
        float2 v[B], o[S][16];
#pragma unroll
        for (int j = 0; j < B; ++j) v[j] = w.hs[w.t + 16 * j];
        __syncwarp(w.mask);
        fft_a<B, true>(v, o, h, tw);
        float2* row = G + t4_row(b, ld);
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (w.t + 16 * s < B) {
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) row[L.at(16 * s + B * k1)] = o[s][k1];
            }
    }
}

// rows of a band of the tiled grid G (ld columns): forward transform along x; returns
// the sum of out(e, value) over this lane's points.
template <int B, int K, class Out>
__device__ __noinline__ float wpass_rows_out(HWw w, const float2* tw, const float2* G, int ld, int nrows,
                                             const int* rp, const int* px, Out out) {
    constexpr int m = 16 * B, S = Slots<B>::value;
    const HalfWarp h = w.h();
    float acc = 0.f;
    const int c0 = t4_col(w.t);
    for (int b = w.gh; b < nrows; b += w.ghs) {
        const float2* row = G + t4_row(b, ld) + c0;
        float2 v[B], o[S][16];
#pragma unroll
        for (int j = 0; j < B; ++j) v[j] = ldx<K>(row + 64 * j);
        // the row's point range and this lane's first point, loaded before the transform
        const int e0 = rp[b] + w.t, e1 = rp[b + 1];
        int xn = e0 < e1 ? px[e0] : 0;
        fft_a<B, false>(v, o, h, tw);
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (w.t + 16 * s < B) {
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) w.hs[w.t + 16 * s + B * k1] = o[s][k1];
            }
        __syncwarp(w.mask);
        for (int e = e0; e < e1; e += 16) {
            const int xc = xn;
            if (e + 16 < e1) xn = px[e + 16];
            acc += out(e, w.hs[freq_index(xc, m)]);
        }
        __syncwarp(w.mask);
    }
    return acc;
}

// columns x < ncols of a grid whose columns have 16 B points: the ni band rows of the
// tiled grid Gi (ldi columns) are the input at column indices 0..ni - 1, the rest zero;
// inverse along y, mid, and (Mid::kOut) forward along y, column indices 0..no - 1
// stored as the band rows of the tiled grid Go (ldo columns). An input band that
// starts at grid row yi0 and an output band at yo0 are thus transformed as if both
// started at row 0: by the shift theorem that multiplies the inverse transform by
// W^(-yi0 k) and the forward one's input by W^(yo0 k), a ramp W^((yo0 - yi0) k) that
// the stored field (the mid's factor) carries (the column passes of the CG run
// between the U and the Q band in both directions, with the field and its
// conjugate). Each half-warp reads and writes its
// own columns, so Gi and Go may be the same grid. Ends with a tile barrier.
// (Measured and left out: staging strips of 32 columns through shared memory for
// 256-byte row accesses, and issuing the next column's loads before the current
// transform; both slowed the kernel by ~10 %: the first adds block barriers between
// half-warps that otherwise overlap one another's loads and transforms, the second
// spills.)
template <int B, int K, class Mid>
__device__ __noinline__ void wpass_cols(HWw w, const float2* tw, int ncols, const float2* Gi, int ldi, int ni,
                                        float2* Go, int ldo, int no, Mid mid) {
    constexpr int S = Slots<B>::value;
    const HalfWarp h = w.h();
    const int ri = t4_row(w.t, ldi), ro = t4_row(w.t, ldo);      // band row t of the lane
    for (int x = w.gh; x < ncols; x += w.ghs) {
        float2 v[B], o[S][16];
        const float2* gi = Gi + ri + t4_col(x);
#pragma unroll
        for (int j = 0; j < B; ++j)                                  // band row t + 16 j
            v[j] = w.t + 16 * j < ni ? ldx<K>(gi + 16 * j * ldi) : make_float2(0.f, 0.f);
        if constexpr (Mid::kPre) {
            typename Mid::Pre pre;
            mid.load(pre, x, w.t);
            fft_a<B, true>(v, o, h, tw);
            mid.apply(o, pre);
        } else {
            fft_a<B, true>(v, o, h, tw);
            mid(o, x, w.t);
        }
        if constexpr (Mid::kOut) {
            fft_b<B, false>(o, v, h, tw);
            float2* go = Go + ro + t4_col(x);
#pragma unroll
            for (int k1 = 0; k1 < B; ++k1)
                if (w.t + 16 * k1 < no) go[16 * k1 * ldo] = v[k1];
        }
    }
    tile_sync<K>();
}

// rows of Q in place (tiled grid of 16 B columns): forward along x, keep the Q lags, inverse
// along x. qmask: per band row 16 words; the bit k1 of half (t + 16 s) & 1 of word
// (t + 16 s) >> 1 says whether x index (t + 16 s) + B k1 is in Q. Ends with __syncthreads.
template <int B, int K>
__device__ __noinline__ void wpass_rows_mask(HWw w, const float2* tw, float2* G, int nrows, const unsigned* qmask) {
    constexpr int m = 16 * B, S = Slots<B>::value;
    const HalfWarp h = w.h();
    const int c0 = t4_col(w.t);
    for (int b = w.gh; b < nrows; b += w.ghs) {
        float2* row = G + t4_row(b, m) + c0;
        float2 v[B], o[S][16];
#pragma unroll
        for (int j = 0; j < B; ++j) v[j] = ldx<K>(row + 64 * j);
        unsigned qw[S];
#pragma unroll
        for (int s = 0; s < S; ++s) qw[s] = qmask[(size_t)b * kWQWords + ((w.t + 16 * s) >> 1)];
        fft_a<B, false>(v, o, h, tw);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int ls = w.t + 16 * s;
            const unsigned bits = qw[s] >> (16 * (ls & 1));
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1)
                if (!((bits >> k1) & 1u)) o[s][k1] = make_float2(0.f, 0.f);
        }
        fft_b<B, true>(o, v, h, tw);
#pragma unroll
        for (int k1 = 0; k1 < B; ++k1) row[64 * k1] = v[k1];
    }
    tile_sync<K>();
}

// Columns of I - |p|^2 (n = 512; the image read transposed with tr, once, with
// evict-first loads): Eq. 13's right-hand side F(I) - P * P is the spectrum of the
// image minus the intensity of the known field, so p's column x is formed from the
// nP band rows of the tiled grid GP (P's rows transformed along x on the camera grid) by an
// inverse transform along y and |p|^2 kept in registers; then the chunk's 32 image
// columns are staged through shared memory (coalesced reads), the difference is
// formed and transformed forward along y; rows qy0.. (nQ) go to GX (row length n).
// Half-warps 0..31 take one column of a chunk each. The stages alias the half-warp
// areas; barriers separate each use from the transforms. Ends with a tile barrier.
template <int K>
__device__ __noinline__ void wpass_image_cols_p(HWw w, const float2* tw, float2* stage, const float* img,
                                                const float2* GP, int nP, float2* GX, int qy0, int nQ,
                                                bool tr) {
    constexpr int BN = kWBN, n = 16 * BN, S = Slots<BN>::value;
    const HalfWarp h = w.h();
    float* stage_f = reinterpret_cast<float*>(stage);
    for (int c0 = 32 * (w.gh / kWHW); c0 < n; c0 += 32 * K) {     // this block's chunks of 32 columns
        const int x = c0 + w.hw;
        float2 v[BN], o[S][16];
        float q[S][16];
        // the band as if it started at row 0: that multiplies p by a phase ramp along
        // y, which |p|^2 does not see
        const float2* gp = GP + t4_row(w.t, n) + t4_col(x);
#pragma unroll
        for (int j = 0; j < BN; ++j) v[j] = w.t + 16 * j < nP ? ldx<K>(gp + 16 * j * n) : make_float2(0.f, 0.f);
        fft_a<BN, true>(v, o, h, tw);               // p(x, y), y = (t + 16 s) + BN k1
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) q[s][k1] = cabs2(o[s][k1]);
        __syncthreads();                            // transforms done: the stage may overwrite the areas
        if (tr) {   // column c of the solve frame is image row c
            for (int idx = threadIdx.x; idx < n * 32; idx += blockDim.x) {
                const int c = idx / n, y = idx - c * n;
                stage_f[y * kWStageLd + c] = __ldcs(img + (size_t)(c0 + c) * n + y);
            }
        } else {
            for (int idx = threadIdx.x; idx < n * 32; idx += blockDim.x) {
                const int y = idx >> 5, c = idx & 31;
                stage_f[y * kWStageLd + c] = __ldcs(img + (size_t)y * n + c0 + c);
            }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                const int y = (w.t + 16 * s < BN ? w.t + 16 * s : 0) + BN * k1;
                o[s][k1] = make_float2(stage_f[y * kWStageLd + w.hw] - q[s][k1], 0.f);
            }
        __syncthreads();                            // the stage is consumed
        fft_b<BN, false>(o, v, h, tw);              // along y: v[k1] at ky = t + 16 k1
        __syncthreads();
#pragma unroll
        for (int k1 = 0; k1 < BN; ++k1) {
            const int bb = sfreqw(w.t + 16 * k1, n) - qy0;
            if (bb >= 0 && bb < nQ) stage[bb * kWStageLd + w.hw] = v[k1];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < nQ * 32; idx += blockDim.x) {
            const int b = idx >> 5, c = idx & 31;
            GX[(size_t)b * n + c0 + c] = stage[b * kWStageLd + c];
        }
        __syncthreads();
    }
    tile_sync<K>();
}

// rows of GX (length n): forward along x, bq[e] = value / n^2 at the Q points. Ends
// with __syncthreads.
template <int K>
__device__ __noinline__ void wpass_image_rows(HWw w, const float2* tw, const float2* GX, int nQ, const int* qrp,
                                              const int* Qx, float2* bq) {
    constexpr int BN = kWBN, n = 16 * BN, S = Slots<BN>::value;
    const HalfWarp h = w.h();
    const float inv_n2 = 1.f / (float)(n * n);
    for (int b = w.gh; b < nQ; b += w.ghs) {
        const float2* row = GX + (size_t)b * n;
        float2 v[BN], o[S][16];
#pragma unroll
        for (int j = 0; j < BN; ++j) v[j] = ldx<K>(row + w.t + 16 * j);
        fft_a<BN, false>(v, o, h, tw);
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (w.t + 16 * s < BN) {
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) w.hs[w.t + 16 * s + BN * k1] = o[s][k1];
            }
        __syncwarp(w.mask);
        for (int e = qrp[b] + w.t; e < qrp[b + 1]; e += 16) bq[e] = cscale(w.hs[freq_index(Qx[e], n)], inv_n2);
        __syncwarp(w.mask);
    }
    tile_sync<K>();
}

}  // namespace

// Shared memory of one block (bytes, 16-aligned offsets):
//   [0, vec)          half-warp areas of the CG grids (17 x 20 values each)
//   [vec, vec_end)    CG vectors x, d, s, w (max_N each)
//   [0, setup)        during an image's setup: half-warp areas of the 512-point
//                     transforms (17 x 32 values each), or the 32-column image
//                     stage, or the output stage of the image columns
//   [tw, tw_end)      step twiddles of the camera grid and of the image's row and
//                     column grids
//   [red, total)      96 doubles of reductions (block partials, then the blocks' totals)
struct DFWSmem {
    size_t vec, tw, red, total;
};

__host__ __device__ inline size_t walign16(size_t b) { return (b + 15) & ~(size_t)15; }

// band: the most band rows a column pass stages (max of the U, P and Q bands)
__host__ __device__ inline DFWSmem dfw_smem_layout(int max_N, int band) {
    DFWSmem L;
    L.vec = walign16(std::max((size_t)kWHW * hw_single_size(kWMaxB), (size_t)band * kWStageLd) * sizeof(float2));
    const size_t cg_end = L.vec + walign16((size_t)4 * max_N * sizeof(float2));
    const size_t setup_hw = (size_t)kWHW * hw_single_size(kWBN) * sizeof(float2);
    const size_t stage_c = (size_t)band * kWStageLd * sizeof(float2);
    const size_t stage_f = (size_t)16 * kWBN * kWStageLd * sizeof(float);
    const size_t setup = std::max(setup_hw, std::max(stage_c, stage_f));
    L.tw = walign16(std::max(cg_end, setup));
    L.red = walign16(L.tw + (size_t)2 * 16 * (kWBN + 2 * kWMaxB) * sizeof(float2));
    L.total = walign16(L.red + 96 * sizeof(double));
    return L;
}

size_t dfw_smem_bytes(int max_N, int band) { return dfw_smem_layout(max_N, band).total; }

// Global scratch of one block: GQ (Q or P band rows on the camera grid), PF (the
// column-major known field of the CG grid, or the image's Q rows), GU (U band rows
// of the CG grid), b on Q.
size_t dfw_scratch_bytes(const DevPlan& P) {
    const int n = P.h;
    size_t s = (size_t)t4_rows(std::max(P.band_q, P.band_p)) * n;                         // GQ (tiled)
    s += std::max((size_t)P.max_mxy, (size_t)P.band_q * n);                               // PF / F(I) rows
    s += (size_t)t4_rows(P.band_u) * P.max_mx;                                            // GU (tiled)
    s += (size_t)P.max_M;                                                                 // b on Q
    return (s * sizeof(float2) + 255) & ~(size_t)255;
}

namespace {

struct DFWCtx {
    HWw w;                  // half-warp areas of the CG grids
    HWw ws;                 // half-warp areas of the 512-point setup transforms
    const float2* tw_n;     // step twiddles of the camera grid
    float2* tw_x;           // step twiddles of the image's row grid (filled per image)
    float2* tw_y;           // step twiddles of the image's column grid (filled per image)
    float2 *GU, *GQ, *PF, *bq;
    float2 *dv, *sv, *wv, *xv;
    float2* stage;          // stages of the setup column pass (alias the half-warp areas)
    double* red;
};

// plain twiddle table of a 16 G-point grid of the wide solve
__device__ __forceinline__ const float2* wgrid_table(const DevPlan& P, int G) {
    return G == 12 ? P.tw_w12 : G == 16 ? P.tw_w16 : G == 18 ? P.tw_w18 : P.tw_w20;
}

// Solve of one darkfield image (image `img`) on a grid of 16 BX row points x 16 BY
// column points, by the K blocks of the cluster: b = F(I - |p|^2) on Q on the camera
// grid, then CGNR. Returns the CG iterations (negative: did not converge).
template <int BX, int BY, int K>
__device__ __forceinline__ int dfw_solve(const DFWCtx& c, const DevPlan& P, const DevDF& D, const float* img,
                                         float2* sp, const float* ph, int iters, float tol) {
    constexpr int n = 16 * kWBN, mx = 16 * BX;
    const HWw& w = c.w;
    const int u_off = D.u_off, p_off = D.p_off, q_off = D.q_off;
    const int uy0 = D.uy0, qy0 = D.qy0, py0 = D.py0;
    const int nU = D.uy1 - uy0 + 1, nQ = D.qy1 - qy0 + 1, nP = D.py1 - py0 + 1;
    const int *urp = P.d_rowptr + D.urp, *qrp = P.d_rowptr + D.qrp, *prp = P.d_rowptr + D.prp;
    const unsigned* qmask = P.d_qmask + D.qmask_off;
    const WValKnown<K> pval{sp, ph, P.dP_ap + p_off, P.dP_pup + p_off};
    make_step_twiddles(c.tw_x, wgrid_table(P, BX), BX);
    make_step_twiddles(c.tw_y, wgrid_table(P, BY), BY);
    __syncthreads();
    // b = F(I) - P * P on Q (Eq. 13) as the spectrum of I - |p|^2 on the camera grid
    // (exact: P * P's lags reach 2 R < n / 2): the known field's band rows along x,
    // then per column p, the difference and its forward transform, then the rows
    wpass_rows_in<kWBN>(c.ws, c.tw_n, c.GQ, n, nP, prp, P.dP_x + p_off, pval);
    tile_sync<K>();
    wpass_image_cols_p<K>(c.ws, c.tw_n, c.stage, img, c.GQ, nP, c.PF, qy0, nQ, D.tr != 0);
    wpass_image_rows<K>(c.ws, c.tw_n, c.PF, nQ, qrp, P.dQ_x + q_off, c.bq);
    // band rows of the known field P (Eq. 11) along x on the row grid, then p s on
    // the column grid, column-major in PF (s = 1 / (mx my): the two unnormalised
    // transforms around each product)
    const float scale = 1.f / ((float)mx * (float)(16 * BY));
    wpass_rows_in<BX>(w, c.tw_x, c.GQ, mx, nP, prp, P.dP_x + p_off, pval);
    tile_sync<K>();
    // the field carries the ramp W^((uy0 - qy0) k) of the U <-> Q column passes and
    // W^(-py0 k) for its own band's start (see wpass_cols)
    const int my = 16 * BY, shift = (((uy0 - qy0 - py0) % my) + my) % my;
    wpass_cols<BY, K>(w, c.tw_y, mx, c.GQ, mx, nP, c.GQ, mx, 0,
                      WMidStoreField<BY>{c.PF, scale, wgrid_table(P, BY), shift});
    // rows of b inverse along x on the row grid; s = d = C^H b
    wpass_rows_in<BX>(w, c.tw_x, c.GQ, mx, nQ, qrp, P.dQ_x + q_off, WValB{c.bq});
    tile_sync<K>();
    wpass_cols<BY, K>(w, c.tw_y, mx, c.GQ, mx, nQ, c.GU, mx, nU, WMidTimesField<BY, false>{c.PF});
    const float g0 =
        wpass_rows_out<BX, K>(w, c.tw_x, c.GU, mx, nU, urp, P.dU_x + u_off, WOutStart{c.sv, c.dv, c.xv});
    int par = 0;
    const double gamma0 = tile_sum<K>(g0, c.red, par);
    // CGNR; each block updates the vector entries of its own U rows
    double gamma = gamma0;
    bool conv = !(gamma0 > 1e-300);
    const double stop = (double)tol * (double)tol * gamma0;
    int it = 0;
    float bf = 0.f;
    for (; it < iters && !conv; ++it) {
        wpass_rows_in<BX>(w, c.tw_x, c.GU, mx, nU, urp, P.dU_x + u_off, WValNextDir{c.sv, c.dv, bf});
        tile_sync<K>();
        wpass_cols<BY, K>(w, c.tw_y, mx, c.GU, mx, nU, c.GQ, mx, nQ, WMidTimesField<BY, true>{c.PF});
        wpass_rows_mask<BX, K>(w, c.tw_x, c.GQ, nQ, qmask);
        wpass_cols<BY, K>(w, c.tw_y, mx, c.GQ, mx, nQ, c.GU, mx, nU, WMidTimesField<BY, false>{c.PF});
        const float dw = wpass_rows_out<BX, K>(w, c.tw_x, c.GU, mx, nU, urp, P.dU_x + u_off, WOutDot{c.wv, c.dv});
        const double delta = tile_sum<K>(dw, c.red, par);
        if (!(delta > 0)) break;
        const double alpha = gamma / delta;
        const float af = (float)alpha;
        float g2 = 0.f;
        auto update = [&](int e) {
            const float2 d = c.dv[e];
            float2 x = c.xv[e];
            x.x += af * d.x;
            x.y += af * d.y;
            c.xv[e] = x;
            const float2 sv = csub(c.sv[e], cscale(c.wv[e], af));
            c.sv[e] = sv;
            g2 += sv.x * sv.x + sv.y * sv.y;
        };
        if constexpr (K == 1) {           // all entries are this block's: every thread an even share
            for (int e = threadIdx.x; e < D.N; e += blockDim.x) update(e);
        } else {                          // the entries of this block's U rows
            for (int b = w.gh; b < nU; b += w.ghs)
                for (int e = urp[b] + w.t; e < urp[b + 1]; e += 16) update(e);
        }
        const double gnew = tile_sum<K>(g2, c.red, par);
        bf = (float)(gnew / gamma);
        gamma = gnew;
        conv = gnew <= stop;
    }
    // corrected unknown spectrum into the tile's spectrum (this block's U rows)
    const int* Upup = P.dU_pup + u_off;
    const int* Uap = P.dU_ap + u_off;
    auto put = [&](int e) {
        float sn, cs;
        sincosf(ph[Upup[e]], &sn, &cs);
        sp[Uap[e]] = cmul(c.xv[e], make_float2(cs, -sn));
    };
    if constexpr (K == 1) {
        for (int e = threadIdx.x; e < D.N; e += blockDim.x) put(e);
    } else {
        for (int b = w.gh; b < nU; b += w.ghs)
            for (int e = urp[b] + w.t; e < urp[b + 1]; e += 16) put(e);
    }
    tile_sync<K>();
    return conv ? it : -1 - it;
}

template <int K>
__global__ void __launch_bounds__(kWThreads, 1)
k_darkfield_wide(DevPlan P, int n_tiles, const float* __restrict__ I, const float* __restrict__ phi,
                 float2* __restrict__ spec, char* __restrict__ scratch, size_t per_block, int iters, float tol,
                 int32_t* __restrict__ status, unsigned long long* __restrict__ counters, int* __restrict__ work) {
    constexpr int n = 16 * kWBN;
    extern __shared__ float4 smem4[];
    char* sbase = reinterpret_cast<char*>(smem4);
    const DFWSmem SL = dfw_smem_layout(P.max_N, max(P.band_q, max(P.band_p, P.band_u)));
    DFWCtx c;
    c.dv = reinterpret_cast<float2*>(sbase + SL.vec);
    c.sv = c.dv + P.max_N;
    c.wv = c.sv + P.max_N;
    c.xv = c.wv + P.max_N;
    c.stage = reinterpret_cast<float2*>(sbase);
    float2* tw_n = reinterpret_cast<float2*>(sbase + SL.tw);
    c.tw_n = tw_n;
    c.tw_x = tw_n + 2 * 16 * kWBN;
    c.tw_y = c.tw_x + 2 * 16 * kWMaxB;
    c.red = reinterpret_cast<double*>(sbase + SL.red);
    make_step_twiddles(tw_n, P.tw_n, kWBN);

    const int rank = K > 1 ? (int)cta_rank() : 0;
    const int slot = blockIdx.x / K, nslots = gridDim.x / K;      // tile slot = the cluster
    c.w.hw = c.ws.hw = threadIdx.x >> 4;
    c.w.gh = c.ws.gh = rank * kWHW + c.w.hw;
    c.w.ghs = c.ws.ghs = K * kWHW;
    c.w.t = c.ws.t = threadIdx.x & 15;
    c.w.mask = c.ws.mask = (threadIdx.x & 16) ? 0xFFFF0000u : 0x0000FFFFu;
    c.w.hs = reinterpret_cast<float2*>(sbase) + c.w.hw * hw_single_size(kWMaxB);
    c.ws.hs = reinterpret_cast<float2*>(sbase) + c.ws.hw * hw_single_size(kWBN);

    char* base = scratch + (size_t)slot * per_block;
    c.GQ = reinterpret_cast<float2*>(base);
    c.PF = c.GQ + (size_t)t4_rows(max(P.band_q, P.band_p)) * n;
    c.GU = c.PF + max((size_t)P.max_mxy, (size_t)P.band_q * n);
    c.bq = c.GU + (size_t)t4_rows(P.band_u) * P.max_mx;
    tile_sync<K>();

    // one block per tile: tiles taken one at a time from the launch's counter (a block that
    // meets skipped background tiles goes on to the next, so uneven batches balance);
    // clusters (and launches without a counter): by stride
    __shared__ int s_next;
    auto take = [&](int prev) -> int {
        if (K > 1 || !work) return prev < 0 ? slot : prev + nslots;
        __syncthreads();
        if (threadIdx.x == 0) s_next = atomicAdd(work, 1);
        __syncthreads();
        return s_next;
    };
    for (int tile = take(-1); tile < n_tiles; tile = take(tile)) {
        if (status && (status[tile] & (APIC_TILE_BACKGROUND | APIC_TILE_BADINPUT))) continue;
        const float* ph = phi + (size_t)tile * P.npup;
        float2* sp = spec + (size_t)tile * P.nap;
        bool notconv = false;
        for (int di = 0; di < P.n_used; ++di) {
            const DevDF& D = P.df[di];
            const float* img = I + ((size_t)tile * P.n_img + D.led) * n * n;
            int r;
            switch (16 * D.bx + D.by) {
                case 16 * 18 + 12: r = dfw_solve<18, 12, K>(c, P, D, img, sp, ph, iters, tol); break;
                case 16 * 18 + 16: r = dfw_solve<18, 16, K>(c, P, D, img, sp, ph, iters, tol); break;
                case 16 * 18 + 18: r = dfw_solve<18, 18, K>(c, P, D, img, sp, ph, iters, tol); break;
                case 16 * 20 + 12: r = dfw_solve<20, 12, K>(c, P, D, img, sp, ph, iters, tol); break;
                case 16 * 20 + 16: r = dfw_solve<20, 16, K>(c, P, D, img, sp, ph, iters, tol); break;
                case 16 * 20 + 18: r = dfw_solve<20, 18, K>(c, P, D, img, sp, ph, iters, tol); break;
                default: r = dfw_solve<20, 20, K>(c, P, D, img, sp, ph, iters, tol); break;
            }
            if (r < 0) notconv = true;
            if (threadIdx.x == 0 && rank == 0 && counters) {
                atomicAdd(counters + 1, (unsigned long long)(r < 0 ? -1 - r : r));
                atomicAdd(counters + 2, 1ull);
                if (di < kCountedImages) atomicAdd(counters + 4 + di, (unsigned long long)(r < 0 ? -1 - r : r));
            }
        }
        if (threadIdx.x == 0 && rank == 0 && notconv && status) atomicOr(status + tile, APIC_TILE_NOTCONV);
    }
}

}  // namespace

using DFWKernel = void (*)(DevPlan, int, const float*, const float*, float2*, char*, size_t, int, float, int32_t*,
                           unsigned long long*, int*);

static DFWKernel dfw_kernel(int K) {
    switch (K) {
        case 1: return k_darkfield_wide<1>;
        case 2: return k_darkfield_wide<2>;
        case 4: return k_darkfield_wide<4>;
        default: return nullptr;
    }
}

// Tile slots (clusters of K blocks) that run at once, 0 on error.
int configure_dfw(size_t smem, int K) {
    DFWKernel f = dfw_kernel(K);
    if (!f || raise_smem_limit((const void*)f, smem) != cudaSuccess) return 0;
    if (K == 1) {
        int occ = 0, dev = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kWThreads, smem) != cudaSuccess) return 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        return occ * sms;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(K * 256, 1, 1);
    cfg.blockDim = dim3(kWThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, f, &cfg) != cudaSuccess) return 0;
    return clusters;
}

// grid: tile slots (clusters); each gets K blocks.
cudaError_t launch_darkfield_wide(const DevPlan& P, int K, int grid, size_t smem, int n_tiles, const float* I,
                                  const float* phi, float2* spec, void* scratch, size_t per_block, int iters,
                                  float tol, int32_t* status, unsigned long long* counters, int* work,
                                  cudaStream_t st) {
    DFWKernel f = dfw_kernel(K);
    if (!f || P.h != 16 * kWBN || P.w != P.h) return cudaErrorInvalidValue;
    const int slots = min(grid, n_tiles);
    if (slots < 1) return cudaErrorInvalidConfiguration;
    if (K == 1) {
        if (work) {
            const cudaError_t e = cudaMemsetAsync(work, 0, sizeof(int), st);
            if (e != cudaSuccess) return e;
        }
        f<<<slots, kWThreads, smem, st>>>(P, n_tiles, I, phi, spec, (char*)scratch, per_block, iters, tol, status,
                                          counters, work);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(K * slots, 1, 1);
    cfg.blockDim = dim3(kWThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, f, P, n_tiles, I, phi, spec, (char*)scratch, per_block, iters, tol, status,
                              counters, (int*)nullptr);
}

}  // namespace apic
