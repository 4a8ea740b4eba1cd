// kernels_dfr.cu - darkfield spectrum extension (WSI-APIC Eq. 11-13) with
// register-resident half-warp FFTs.
//
// Per darkfield image j (pupil frame c = K + k_j; U unknown, P known, Q lags):
//   b(k) = F(I_j)(k) - (P*P)(k) on Q                              (Eq. 13 left)
//   C u  = series coefficients on Q of u(x) conj p(x)              (Eq. 13 right)
//   min ||C u - b|| by CG on the normal equations C^H C u = C^H b (CGNR): per
//   iteration w = C^H mask_Q C d as five passes over an mx x my grid
//     R1 rows of U: scatter d, inverse transform along x     -> GU
//     C1 columns:   inverse along y, * conj(p) / (mx my), forward along y -> GQ
//     R2 rows of Q: forward along x, keep Q, inverse along x (in place)
//     C2 columns:   inverse along y, * p / (mx my), forward along y       -> GU
//     R3 rows of U: forward along x, gather w on U, <d, w>
//   then x += alpha d, s -= alpha w, and d = s + beta d (folded into the next
//   R1). Transforms, vectors and the partial sums of a thread and of a warp FP32;
//   the sums across warps and the step lengths FP64 (the FP64 pipe is narrow, so it
//   sees 16 values per reduction rather than every point).
// Each image is solved in its own frame (x and y swapped when that makes the row
// bands shorter) on its own grid: mx = 16 BX row points and my = 16 BY column
// points, the cheapest supported pair on which both correlations are exact
// (chosen with the plan); P * P, whose lags reach further, uses the m x m grid
// (m = 16 B). Columns of <= 128 points go two per half-warp (all 16 lanes in the
// DFT_16 step), longer ones two per half-warp in turn; column pairs of grids with
// an even row stride move as one 16-byte access per row. The known field p of the
// paired grids lives in tensor memory (each thread's own lane and columns).
// GU / GQ are band-row grids (only rows holding U or Q points). GU and the CG
// vectors (the solution included) live in shared memory (GU with row stride
// gu_ld(B): column passes are conflict free per warp - m + 2 where they move column
// pairs as 16-byte accesses, m + 1 where single columns); GQ, the column-major known
// field p of the longer grids and b on Q live in the block's global scratch
// (L2-resident; data read once - the images - is loaded evict-first). The setup
// transforms of each image reuse the shared-memory space of GU. One block per tile
// (persistent); images of a tile are sequential. Each pass is a separate
// (non-inlined) function so registers are allocated per pass.
#include <math.h>

#include <algorithm>

#include "../../include/apic.h"
#include "internal.cuh"
#include "regfft.cuh"

namespace apic {

namespace {

#ifndef APIC_DF_THREADS
#define APIC_DF_THREADS 512
#endif

constexpr int kDFThreads = APIC_DF_THREADS;  // threads per block of this kernel
constexpr int kHW = kDFThreads / 16;         // half-warps per block
constexpr int kStageLd = 33;           // column stage: 32 columns + 1 pad

__device__ __forceinline__ int sfreq(int i, int n) { return i < n / 2 ? i : i - n; }

// ---- tensor memory as per-thread storage of the known field
// The darkfield kernel issues no MMA; its 512 TMEM columns x 128 lanes (256 KB per
// SM) hold each thread's share of the column-major known field p on the paired
// column grids. Thread i of warp w owns lane 32 (w mod 4) + i and the
// kTmemSlotCols columns of slot floor(w / 4): 16 complex values (32 columns) per
// column pair it transforms. A thread reads back only what it stored itself.
constexpr int kTmemCols = 512;
constexpr int kTmemSlots = kDFThreads / 128;                  // warps per lane quarter
constexpr int kTmemSlotCols = kTmemSlots > 0 ? (kTmemCols / kTmemSlots) & ~31 : 0;
// every pass has at most 3 pair rounds (<= 96 pairs of columns over >= 32 half-warps)
constexpr bool kTmemField = kDFThreads % 128 == 0 && kTmemSlotCols >= 96;

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float2 (&v)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
                 :: "r"(taddr), "f"(v[0].x), "f"(v[0].y), "f"(v[1].x), "f"(v[1].y), "f"(v[2].x), "f"(v[2].y), "f"(v[3].x), "f"(v[3].y), "f"(v[4].x), "f"(v[4].y), "f"(v[5].x), "f"(v[5].y), "f"(v[6].x), "f"(v[6].y), "f"(v[7].x), "f"(v[7].y), "f"(v[8].x), "f"(v[8].y), "f"(v[9].x), "f"(v[9].y), "f"(v[10].x), "f"(v[10].y), "f"(v[11].x), "f"(v[11].y), "f"(v[12].x), "f"(v[12].y), "f"(v[13].x), "f"(v[13].y), "f"(v[14].x), "f"(v[14].y), "f"(v[15].x), "f"(v[15].y) : "memory");
}
// load and wait in one statement, so no use of v can be scheduled before the wait
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float2 (&v)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y), "=f"(v[2].x), "=f"(v[2].y), "=f"(v[3].x), "=f"(v[3].y), "=f"(v[4].x), "=f"(v[4].y), "=f"(v[5].x), "=f"(v[5].y), "=f"(v[6].x), "=f"(v[6].y), "=f"(v[7].x), "=f"(v[7].y), "=f"(v[8].x), "=f"(v[8].y), "=f"(v[9].x), "=f"(v[9].y), "=f"(v[10].x), "=f"(v[10].y), "=f"(v[11].x), "=f"(v[11].y), "=f"(v[12].x), "=f"(v[12].y), "=f"(v[13].x), "=f"(v[13].y), "=f"(v[14].x), "=f"(v[14].y), "=f"(v[15].x), "=f"(v[15].y) : "r"(taddr) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

struct HW {
    int t, hw;
    unsigned mask;
    float2* hs;
    __device__ HalfWarp h() const { return HalfWarp{t, mask, hs}; }
};

// ---- per-point functors
struct ValKnown {       // P(c) = O_known(K) exp(j phi(c))
    const float2* sp;
    const float* ph;
    const int* ap;
    const int* pup;
    __device__ float2 operator()(int e) const {
        float sn, cs;
        sincosf(ph[pup[e]], &sn, &cs);
        return cmul(sp[ap[e]], make_float2(cs, sn));
    }
};
struct ValNextDir {     // d = s + beta d (stored back), scattered into the rows
    const float2* sv;
    float2* dv;
    float beta;
    __device__ float2 operator()(int e) const {
        const float2 d = cadd(sv[e], cscale(dv[e], beta));
        dv[e] = d;
        return d;
    }
};
struct OutStart {       // s = d = C^H b, x = 0; returns |s|^2
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
struct ValB {           // b on Q
    const float2* bq;
    __device__ float2 operator()(int e) const { return bq[e]; }
};
struct OutDot {         // w = C^H C d; returns Re <d, w>
    float2* wv;
    const float2* dv;
    __device__ float operator()(int e, float2 v) const {
        wv[e] = v;
        const float2 d = dv[e];
        return d.x * v.x + d.y * v.y;
    }
};

// ---- per-column mid operations (lanes t < B; o[k1] is the value at y = t + B k1)
template <int B>
struct MidStoreField {  // store p s W^(shift y) (p scaled; wt: W_16B^j) column-major (16 B per column)
    float2* PF;
    float scale;
    const float2* wt;
    int shift;
    static constexpr bool kReadsField = false, kTmem = false;
    __device__ void operator()(float2 (&o)[16], int x, int t, const float2 (&)[16]) const {
        float2* col = PF + (size_t)x * (16 * B);
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) {
            const int y = t + B * k1;
            col[y] = cscale(cmul(o[k1], wt[(shift * y) % (16 * B)]), scale);
        }
    }
};
template <int B>
struct MidAbs2 {        // replace p by |p|^2 W^(shift y) (wt: W_16B^j)
    float2* PF = nullptr;
    const float2* wt;
    int shift;
    static constexpr bool kReadsField = false, kTmem = false;
    __device__ void operator()(float2 (&o)[16], int, int t, const float2 (&)[16]) const {
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) o[k1] = cscale(wt[(shift * (t + B * k1)) % (16 * B)], cabs2(o[k1]));
    }
};
template <int B, bool CONJ>
struct MidTimesField {  // o *= p s or conj(p s), p s = the stored, scaled field (loaded by the caller)
    const float2* PF;
    static constexpr bool kReadsField = true, kTmem = false;
    __device__ void operator()(float2 (&o)[16], int x, int t, const float2 (&pf)[16]) const {
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) o[k1] = CONJ ? cmulc(o[k1], pf[k1]) : cmul(o[k1], pf[k1]);
    }
};
// The same two operations with p in the thread's TMEM columns (paired passes; the
// whole warp calls them, r = the half-warp's column-pair round)
struct MidStoreFieldT {  // p s W^(shift y) (wt: W_16B^j; B of the paired grid)
    uint32_t taddr;
    float scale;
    const float2* wt;
    int shift, B;
    static constexpr bool kReadsField = false, kTmem = true;
    __device__ void tm(float2 (&o)[16], int r) const {
        const int t = threadIdx.x & 15, u = t >= B ? t - B : t, m = 16 * B;   // lane t: point u of its column
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) o[k1] = cscale(cmul(o[k1], wt[(shift * (u + B * k1)) % m]), scale);
        tmem_st16(taddr + 32 * r, o);
    }
};
template <bool CONJ>
struct MidTimesFieldT {
    uint32_t taddr;
    static constexpr bool kReadsField = false, kTmem = true;
    __device__ void tm(float2 (&o)[16], int r) const {
        float2 pf[16];
        tmem_ld16(taddr + 32 * r, pf);
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) o[k1] = CONJ ? cmulc(o[k1], pf[k1]) : cmul(o[k1], pf[k1]);
    }
};

// ---- passes

// rows of a band: scatter val(e) at x = px[e], inverse transform along x, store rows of G (row stride ld)
template <int B, class Val>
__device__ __noinline__ void pass_rows_in(HW w, const float2* tw, float2* G, int ld, int nrows, const int* rp,
                                          const int* px, Val val) {
    constexpr int m = 16 * B;
    const HalfWarp h = w.h();
    for (int b = w.hw; b < nrows; b += kHW) {
#pragma unroll
        for (int j = 0; j < B; ++j) w.hs[w.t + 16 * j] = make_float2(0.f, 0.f);
        __syncwarp(w.mask);
        for (int e = rp[b] + w.t; e < rp[b + 1]; e += 16) w.hs[freq_index(px[e], m)] = val(e);
        __syncwarp(w.mask);
        float2 v[B], o[16];
#pragma unroll
        for (int j = 0; j < B; ++j) v[j] = w.hs[w.t + 16 * j];
        __syncwarp(w.mask);
        fft_alpha<B, true>(v, o, h, tw);
        if (w.t < B) {
            float2* row = G + (size_t)b * ld;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) row[w.t + B * k1] = o[k1];
        }
    }
}

// rows of a band of G: forward transform along x; returns sum of out(e, value) over this lane's points
template <int B, class Out>
__device__ __noinline__ float pass_rows_out(HW w, const float2* tw, const float2* G, int ld, int nrows,
                                             const int* rp, const int* px, Out out) {
    constexpr int m = 16 * B;
    const HalfWarp h = w.h();
    float acc = 0.f;
    for (int b = w.hw; b < nrows; b += kHW) {
        const float2* row = G + (size_t)b * ld;
        float2 v[B], o[16];
#pragma unroll
        for (int j = 0; j < B; ++j) v[j] = row[w.t + 16 * j];
        fft_alpha<B, false>(v, o, h, tw);
        if (w.t < B) {
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) w.hs[w.t + B * k1] = o[k1];
        }
        __syncwarp(w.mask);
        for (int e = rp[b] + w.t; e < rp[b + 1]; e += 16) acc += out(e, w.hs[freq_index(px[e], m)]);
        __syncwarp(w.mask);
    }
    return acc;
}

// columns x < ncols of a grid whose columns have 16 B points: the ni band rows of Gi
// (row stride ldi) are the input at column indices 0..ni - 1, the rest zero; inverse
// along y, mid, forward along y; column indices 0..no - 1 stored as the band rows of
// Go (row stride ldo; no = 0: nothing stored, no forward transform). A band that
// starts at grid row y0 is thus transformed as if it started at row 0; by the shift
// theorem the mid's factor carries the ramp W^((yo0 - yi0) y) (the stored field for
// the CG's U <-> Q passes in both directions, see df_solve). Each half-warp reads
// and writes its own columns, so Gi and Go may be the same grid; the known-field
// values of the column are loaded after the first transform. Ends with
// __syncthreads.
template <int B, class Mid>
__device__ __noinline__ void pass_cols(HW w, const float2* tw, int ncols, const float2* Gi, int ldi, int ni,
                                       float2* Go, int ldo, int no, Mid mid) {
    static_assert(!Mid::kTmem, "TMEM operations need the paired pass");
    constexpr int m = 16 * B;
    const HalfWarp h = w.h();
    for (int x = w.hw; x < ncols; x += kHW) {
        float2 v[B], o[16], pf[16];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int bb = w.t + 16 * j;
            v[j] = bb < ni ? Gi[(size_t)bb * ldi + x] : make_float2(0.f, 0.f);
        }
        fft_alpha<B, true>(v, o, h, tw);
        // the known field of the column, loaded once the inputs are consumed (loading it
        // up front with the inputs keeps 32 more registers live through the transform and
        // measured 4 % slower)
        if (Mid::kReadsField && w.t < B) {
            const float2* col = mid.PF + (size_t)x * m;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) pf[k1] = col[w.t + B * k1];
        }
        if (w.t < B) mid(o, x, w.t, pf);
        if (no > 0) {
            fft_beta<B, false>(o, v, h, tw);
#pragma unroll
            for (int k1 = 0; k1 < B; ++k1) {
                const int bb = w.t + 16 * k1;
                if (bb < no) Go[(size_t)bb * ldo + x] = v[k1];
            }
        }
    }
    __syncthreads();
}

// pass_cols for short columns (2 B <= 16): each half-warp transforms the column pair
// x, x + 1 together (fft_alpha2 / fft_beta2), so every lane works in the DFT_16 step
// and each pass makes half as many round trips per half-warp. ncols is even; a grid
// with an even row stride (16-byte aligned rows) moves each pair as one 16-byte access.
template <int B, class Mid>
__device__ __noinline__ void pass_cols2(HW w, const float2* tw, int ncols, const float2* Gi, int ldi, int ni,
                                        float2* Go, int ldo, int no, Mid mid) {
    constexpr int m = 16 * B;
    const HalfWarp h = w.h();
    const int side = w.t >= B ? 1 : 0;           // lanes t < 2 B: column x + side, point u
    const int u = w.t - side * B;
    // both half-warps of a warp take the same number of rounds (ncols / 2 = 8 B is even),
    // so the warp is converged at the TMEM accesses
    int r = 0;
    const bool vin = (ldi & 1) == 0, vout = (ldo & 1) == 0;
    for (int x = 2 * w.hw; x < ncols; x += 2 * kHW, ++r) {
        float2 va[B], vb[B], o[16], pf[16];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int bb = w.t + 16 * j;
            if (bb < ni) {
                const float2* g = Gi + (size_t)bb * ldi + x;
                if (vin) {
                    const float4 q = *reinterpret_cast<const float4*>(g);
                    va[j] = make_float2(q.x, q.y);
                    vb[j] = make_float2(q.z, q.w);
                } else {
                    va[j] = g[0];
                    vb[j] = g[1];
                }
            } else {
                va[j] = vb[j] = make_float2(0.f, 0.f);
            }
        }
        fft_alpha2<B, true>(va, vb, o, h, tw);
        if constexpr (Mid::kTmem) {
            static_assert(!Mid::kReadsField, "a TMEM operation loads its field itself");
            __syncwarp();
            mid.tm(o, r);
        } else {
            if (Mid::kReadsField && w.t < 2 * B) {
                const float2* col = mid.PF + (size_t)(x + side) * m;
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) pf[k1] = col[u + B * k1];
            }
            if (w.t < 2 * B) mid(o, x + side, u, pf);
        }
        if (no > 0) {
            fft_beta2<B, false>(o, va, vb, h, tw);
#pragma unroll
            for (int k1 = 0; k1 < B; ++k1) {
                const int bb = w.t + 16 * k1;
                if (bb < no) {
                    float2* g = Go + (size_t)bb * ldo + x;
                    if (vout) {
                        *reinterpret_cast<float4*>(g) = make_float4(va[k1].x, va[k1].y, vb[k1].x, vb[k1].y);
                    } else {
                        g[0] = va[k1];
                        g[1] = vb[k1];
                    }
                }
            }
        }
    }
    __syncthreads();
}

// pass_cols for columns too long to pair in the lanes (B > 8): each half-warp takes the
// column pair x, x + 1 and transforms the two in turn, so that the pair still moves as
// one 16-byte access per row on grids with an even row stride. ncols is even.
template <int B, class Mid>
__device__ __noinline__ void pass_cols_seq2(HW w, const float2* tw, int ncols, const float2* Gi, int ldi, int ni,
                                            float2* Go, int ldo, int no, Mid mid) {
    static_assert(!Mid::kTmem, "TMEM operations need the paired pass");
    constexpr int m = 16 * B;
    const HalfWarp h = w.h();
    const bool vin = (ldi & 1) == 0, vout = (ldo & 1) == 0;
    for (int x = 2 * w.hw; x < ncols; x += 2 * kHW) {
        float2 va[B], vb[B], o[16], pf[16];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int bb = w.t + 16 * j;
            if (bb < ni) {
                const float2* g = Gi + (size_t)bb * ldi + x;
                if (vin) {
                    const float4 q = *reinterpret_cast<const float4*>(g);
                    va[j] = make_float2(q.x, q.y);
                    vb[j] = make_float2(q.z, q.w);
                } else {
                    va[j] = g[0];
                    vb[j] = g[1];
                }
            } else {
                va[j] = vb[j] = make_float2(0.f, 0.f);
            }
        }
        fft_alpha<B, true>(va, o, h, tw);
        if (Mid::kReadsField && w.t < B) {
            const float2* col = mid.PF + (size_t)x * m;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) pf[k1] = col[w.t + B * k1];
        }
        if (w.t < B) mid(o, x, w.t, pf);
        if (no > 0) fft_beta<B, false>(o, va, h, tw);
        fft_alpha<B, true>(vb, o, h, tw);
        if (Mid::kReadsField && w.t < B) {
            const float2* col = mid.PF + (size_t)(x + 1) * m;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) pf[k1] = col[w.t + B * k1];
        }
        if (w.t < B) mid(o, x + 1, w.t, pf);
        if (no > 0) {
            fft_beta<B, false>(o, vb, h, tw);
#pragma unroll
            for (int k1 = 0; k1 < B; ++k1) {
                const int bb = w.t + 16 * k1;
                if (bb < no) {
                    float2* g = Go + (size_t)bb * ldo + x;
                    if (vout) {
                        *reinterpret_cast<float4*>(g) = make_float4(va[k1].x, va[k1].y, vb[k1].x, vb[k1].y);
                    } else {
                        g[0] = va[k1];
                        g[1] = vb[k1];
                    }
                }
            }
        }
    }
    __syncthreads();
}

// column pass on a 16 B grid: paired columns where two fit a half-warp, column pairs
// in turn up to B = 12, single columns beyond
template <int B, class Mid>
__device__ __forceinline__ void cols(HW w, const float2* tw, int ncols, const float2* Gi, int ldi, int ni,
                                     float2* Go, int ldo, int no, Mid mid) {
    if constexpr (2 * B <= 16)
        pass_cols2<B>(w, tw, ncols, Gi, ldi, ni, Go, ldo, no, mid);
    else if constexpr (B <= 12)
        pass_cols_seq2<B>(w, tw, ncols, Gi, ldi, ni, Go, ldo, no, mid);
    else
        pass_cols<B>(w, tw, ncols, Gi, ldi, ni, Go, ldo, no, mid);
}

// rows of Q in place: forward along x, keep the Q lags, inverse along x. Ends with __syncthreads.
template <int B>
__device__ __noinline__ void pass_rows_mask(HW w, const float2* tw, float2* G, int nrows, const unsigned* qmask) {
    constexpr int m = 16 * B;
    const HalfWarp h = w.h();
    for (int b = w.hw; b < nrows; b += kHW) {
        float2* row = G + (size_t)b * m;
        // lane t's Q membership of x = t + B k1 (bit k1)
        const unsigned bits = qmask[(size_t)b * 8 + (w.t >> 1)] >> (16 * (w.t & 1));
        float2 v[B], o[16];
#pragma unroll
        for (int j = 0; j < B; ++j) v[j] = row[w.t + 16 * j];
        fft_alpha<B, false>(v, o, h, tw);
        if (w.t < B) {
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1)
                if (!((bits >> k1) & 1u)) o[k1] = make_float2(0.f, 0.f);
        }
        fft_beta<B, true>(o, v, h, tw);
#pragma unroll
        for (int k1 = 0; k1 < B; ++k1) row[w.t + 16 * k1] = v[k1];
    }
    __syncthreads();
}

// columns of the real image (n = 16 BN; with tr the transposed image; read once, with
// evict-first loads that leave the L2-resident band grids in place): forward along
// y, rows qy0.. (nQ) stored to GX (row length n). Chunks of 32 columns staged through
// shared memory for coalesced image reads; half-warps 0..31 transform them. Ends with
// __syncthreads.
template <int BN>
__device__ __noinline__ void pass_image_cols(HW w, const float2* tw, float2* stage, const float* img, float2* GX,
                                             int qy0, int nQ, bool tr) {
    constexpr int n = 16 * BN;
    const HalfWarp h = w.h();
    float* stage_f = reinterpret_cast<float*>(stage);
    for (int c0 = 0; c0 < n; c0 += 32) {
        if (tr) {   // image read transposed: column c of the solve frame is image row c
            for (int idx = threadIdx.x; idx < n * 32; idx += blockDim.x) {
                const int c = idx / n, y = idx - c * n;
                stage_f[y * kStageLd + c] = __ldcs(img + (size_t)(c0 + c) * n + y);
            }
        } else {
            for (int idx = threadIdx.x; idx < n * 32; idx += blockDim.x) {
                const int y = idx >> 5, c = idx & 31;
                stage_f[y * kStageLd + c] = __ldcs(img + (size_t)y * n + c0 + c);
            }
        }
        __syncthreads();
        float2 v[BN], o[16];
        if (w.hw < 32) {
#pragma unroll
            for (int j = 0; j < BN; ++j) v[j] = make_float2(stage_f[(w.t + 16 * j) * kStageLd + w.hw], 0.f);
        }
        __syncthreads();
        if (w.hw < 32) {
            fft_alpha<BN, false>(v, o, h, tw);
            if (w.t < BN) {
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) {
                    const int bb = sfreq(w.t + BN * k1, n) - qy0;
                    if (bb >= 0 && bb < nQ) stage[bb * kStageLd + w.hw] = o[k1];
                }
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < nQ * 32; idx += blockDim.x) {
            const int b = idx >> 5, c = idx & 31;
            GX[(size_t)b * n + c0 + c] = stage[b * kStageLd + c];
        }
        __syncthreads();
    }
}

// rows of GX (length n): forward along x, bq[e] = value / n^2 at the Q points. Ends with __syncthreads.
template <int BN>
__device__ __noinline__ void pass_image_rows(HW w, const float2* tw, const float2* GX, int nQ, const int* qrp,
                                             const int* Qx, float2* bq) {
    constexpr int n = 16 * BN;
    const HalfWarp h = w.h();
    const float inv_n2 = 1.f / (float)(n * n);
    for (int b = w.hw; b < nQ; b += kHW) {
        const float2* row = GX + (size_t)b * n;
        float2 v[BN], o[16];
#pragma unroll
        for (int j = 0; j < BN; ++j) v[j] = row[w.t + 16 * j];
        fft_alpha<BN, false>(v, o, h, tw);
        if (w.t < BN) {
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) w.hs[w.t + BN * k1] = o[k1];
        }
        __syncwarp(w.mask);
        for (int e = qrp[b] + w.t; e < qrp[b + 1]; e += 16) bq[e] = cscale(w.hs[freq_index(Qx[e], n)], inv_n2);
        __syncwarp(w.mask);
    }
    __syncthreads();
}

// rows of Q holding the column-transformed |p|^2: forward along x, b = bq - (P*P)/m^2
// on Q (kept in bq), then (INV) the rows of b inverse-transformed along x. Ends with
// __syncthreads.
template <int B, bool INV>
__device__ __noinline__ void pass_rows_rhs(HW w, const float2* tw, float2* GQ, int nQ, const int* qrp,
                                           const int* Qx, float2* bq) {
    constexpr int m = 16 * B;
    const HalfWarp h = w.h();
    const float inv_m2 = 1.f / (float)(m * m);
    for (int b = w.hw; b < nQ; b += kHW) {
        float2* row = GQ + (size_t)b * m;
        float2 v[B], o[16];
#pragma unroll
        for (int j = 0; j < B; ++j) v[j] = row[w.t + 16 * j];
        fft_alpha<B, false>(v, o, h, tw);
        if (w.t < B) {
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) w.hs[w.t + B * k1] = o[k1];
        }
        __syncwarp(w.mask);
        for (int e = qrp[b] + w.t; e < qrp[b + 1]; e += 16)
            bq[e] = csub(bq[e], cscale(w.hs[freq_index(Qx[e], m)], inv_m2));
        __syncwarp(w.mask);
        if constexpr (!INV) continue;
#pragma unroll
        for (int j = 0; j < B; ++j) w.hs[w.t + 16 * j] = make_float2(0.f, 0.f);
        __syncwarp(w.mask);
        for (int e = qrp[b] + w.t; e < qrp[b + 1]; e += 16) w.hs[freq_index(Qx[e], m)] = bq[e];
        __syncwarp(w.mask);
#pragma unroll
        for (int j = 0; j < B; ++j) v[j] = w.hs[w.t + 16 * j];
        __syncwarp(w.mask);
        fft_alpha<B, true>(v, o, h, tw);
        if (w.t < B) {
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) row[w.t + B * k1] = o[k1];
        }
    }
    __syncthreads();
}

}  // namespace

// Shared memory of one block (bytes, 16-aligned offsets):
//   [0, gu)        half-warp areas of the m-grid passes
//   [gu, c)        GU, band_u rows of gu_ld(B) complex values
//   [0, c)         during the setup transforms of an image: half-warp areas of
//                  the n-grid passes, then the column stage (aliases the above)
//   [x, c)         solution x
//   [c, total)     CG vectors d, s, w; step twiddles of m and n; reduction slots
struct DFRSmem {
    size_t gu, stage, x, c, total;
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Half-warp area of the m-grid passes: single transforms of 16 B points and, for
// the column grids of 16 BY points with 2 BY <= 16 (BY = B for B <= 8; 6 or 8 on
// the 192-point grid), column pairs.
__host__ __device__ constexpr int hw_area_m(int B) {
    const int pb = B == 12 ? 8 : (B <= 8 ? B : 0);
    const int p = pb ? hw_pair_size(pb) : 0;
    return hw_single_size(B) > p ? hw_single_size(B) : p;
}

// Row stride of GU (complex values): even (16-byte aligned rows) where the column
// passes move column pairs, odd where they move single columns (B = 16)
__host__ __device__ constexpr int gu_ld(int B) { return B <= 12 ? 16 * B + 2 : 16 * B + 1; }

__host__ __device__ inline DFRSmem dfr_smem_layout(int B, int BN, int band_u, int band_q, int max_N) {
    const int m = 16 * B, n = 16 * BN;
    const int hws_m = hw_area_m(B);
    const int hws_n = hw_single_size(BN);
    DFRSmem L;
    L.gu = align16((size_t)kHW * hws_m * sizeof(float2));
    const size_t gu_end = L.gu + align16((size_t)band_u * gu_ld(B) * sizeof(float2));
    L.stage = align16((size_t)kHW * hws_n * sizeof(float2));
    const size_t stage_c = (size_t)band_q * kStageLd * sizeof(float2);
    const size_t stage_f = (size_t)n * kStageLd * sizeof(float);
    const size_t stage_end = L.stage + align16(stage_c > stage_f ? stage_c : stage_f);
    L.x = gu_end > stage_end ? gu_end : stage_end;
    L.c = L.x + align16((size_t)max_N * sizeof(float2));
    size_t t = L.c + (size_t)3 * max_N * sizeof(float2);                   // d, s, w
    t += (size_t)2 * (m + n) * sizeof(float2);                            // step twiddles
    t += (size_t)4 * m * sizeof(float2);                                  // column- and row-grid step twiddles
    t = align16(t) + 64 * sizeof(double);                                 // reductions
    L.total = align16(t);
    return L;
}

size_t dfr_smem_bytes(int B, int BN, int band_u, int band_q, int max_N) {
    return dfr_smem_layout(B, BN, band_u, band_q, max_N).total;
}

// Global scratch of one block: GQ (Q or P band rows), the known field / image
// rows, b on Q.
size_t dfr_scratch_bytes(const DevPlan& P) {
    const int m = P.mr, n = P.h;
    size_t s = (size_t)(P.band_q > P.band_p ? P.band_q : P.band_p) * m * sizeof(float2);  // GQ
    s += std::max((size_t)m * m, (size_t)P.band_q * n) * sizeof(float2);           // PF / F(I) rows
    s += (size_t)P.max_M * sizeof(float2);                                         // b on Q
    return (s + 255) & ~(size_t)255;
}

// Per-block working set of the darkfield kernel.
struct DFCtx {
    HW w;
    const float2* tw_m;     // step twiddles of the rows (16 B points)
    float2* tw_y;           // step twiddles of the image's column grid (filled per image)
    float2* tw_x;           // step twiddles of the image's row grid (filled per image)
    float2 *GU, *GQ, *PF, *bq;
    float2 *dv, *sv, *wv;
    float2* xv;
    double* red;
    uint32_t tm;            // this thread's TMEM columns (lane and column fields)
};

// Whether a kernel with row grid 16 B has column grids that keep p in TMEM
__host__ __device__ constexpr bool uses_tmem(int B) { return kTmemField && (B == 12 || B <= 8); }

// Column pass that multiplies by the scaled field p s or its conjugate: from TMEM on
// paired grids, else from the column-major copy in global scratch
template <int BY, bool CONJ>
__device__ __forceinline__ void cols_times(const DFCtx& c, const float2* tw, int m, const float2* Gi, int ldi, int ni,
                                           float2* Go, int ldo, int no) {
    if constexpr (2 * BY <= 16 && kTmemField)
        cols<BY>(c.w, tw, m, Gi, ldi, ni, Go, ldo, no, MidTimesFieldT<CONJ>{c.tm});
    else
        cols<BY>(c.w, tw, m, Gi, ldi, ni, Go, ldo, no, MidTimesField<BY, CONJ>{c.PF});
}

// plain twiddle table of a 16 G-point grid of a solve on the 16 B-point register grid
__device__ __forceinline__ const float2* grid_table(const DevPlan& P, int G, int B) {
    return G == B ? P.tw_r : G == 6 ? P.tw_y6 : G == 8 ? P.tw_y8 : G == 9 ? P.tw_y9 : P.tw_y10;
}

// Solve of one darkfield image once b = F(I) on Q is in bq, on a grid of 16 BX rows
// points x 16 BY column points (chosen at plan time, <= 16 B each, as the cheapest on
// which both correlations of Eq. 13 are free of aliasing). P * P, whose lags reach
// further, is formed on the 16 B x 16 B grid. Returns the CG iterations (negative:
// did not converge).
template <int B, int BX, int BY>
__device__ __forceinline__ int df_solve(const DFCtx& c, const DevPlan& P, const DevDF& D, float2* sp, const float* ph,
                                        int iters, float tol) {
    constexpr int m = 16 * B, mx = 16 * BX, my = 16 * BY, LDU = gu_ld(B);
    const HW& w = c.w;
    const int u_off = D.u_off, p_off = D.p_off, q_off = D.q_off;
    const int uy0 = D.uy0, qy0 = D.qy0, py0 = D.py0;
    const int N = D.N, nU = D.uy1 - uy0 + 1, nQ = D.qy1 - qy0 + 1, nP = D.py1 - py0 + 1;
    const int *urp = P.d_rowptr + D.urp, *qrp = P.d_rowptr + D.qrp, *prp = P.d_rowptr + D.prp;
    const unsigned* qmask = P.d_qmask + D.qmask_off;
    const ValKnown pval{sp, ph, P.dP_ap + p_off, P.dP_pup + p_off};
    const float2* twy = c.tw_m;
    if (BY != B) {
        make_step_twiddles(c.tw_y, grid_table(P, BY, B), BY);
        twy = c.tw_y;
    }
    const float2* twx = c.tw_m;
    if (BX != B) {
        make_step_twiddles(c.tw_x, grid_table(P, BX, B), BX);
        twx = c.tw_x;
        __syncthreads();
    }
    // band rows of the known field P (Eq. 11) along x on the row grid, staged in GQ
    // (row stride mx), then p s on the column grid (s = 1 / (mx my): the two
    // unnormalised transforms around each product)
    pass_rows_in<BX>(w, twx, c.GQ, mx, nP, prp, P.dP_x + p_off, pval);
    __syncthreads();
    // (the columns passes transform each band as if it started at row 0, so the field
    // carries the ramp W^((uy0 - qy0) y) of the U <-> Q passes and W^(-py0 y) for its
    // own band's start)
    const float scale = 1.f / ((float)mx * (float)my);
    const int shift = (((uy0 - qy0 - py0) % my) + my) % my;
    if constexpr (2 * BY <= 16 && kTmemField) {
        cols<BY>(w, twy, mx, c.GQ, mx, nP, c.GQ, mx, 0,
                 MidStoreFieldT{c.tm, scale, grid_table(P, BY, B), shift, BY});
        tmem_wait_st();
    } else {
        cols<BY>(w, twy, mx, c.GQ, mx, nP, c.GQ, mx, 0,
                 MidStoreField<BY>{c.PF, scale, grid_table(P, BY, B), shift});
    }
    // |p|^2 (blind to the P band's start) times W^(qy0 y): its transform's Q band from row 0
    const MidAbs2<B> abs2{nullptr, P.tw_r, ((qy0 % m) + m) % m};
    // b -= P * P on Q (16 B grid), then the rows of b inverse along x on the row grid
    if constexpr (BX == B) {
        cols<B>(w, c.tw_m, m, c.GQ, m, nP, c.GQ, m, nQ, abs2);
        pass_rows_rhs<B, true>(w, c.tw_m, c.GQ, nQ, qrp, P.dQ_x + q_off, c.bq);
    } else {
        pass_rows_in<B>(w, c.tw_m, c.GQ, m, nP, prp, P.dP_x + p_off, pval);
        __syncthreads();
        cols<B>(w, c.tw_m, m, c.GQ, m, nP, c.GQ, m, nQ, abs2);
        pass_rows_rhs<B, false>(w, c.tw_m, c.GQ, nQ, qrp, P.dQ_x + q_off, c.bq);
        pass_rows_in<BX>(w, twx, c.GQ, mx, nQ, qrp, P.dQ_x + q_off, ValB{c.bq});
        __syncthreads();
    }
    // s = d = C^H b
    cols_times<BY, false>(c, twy, mx, c.GQ, mx, nQ, c.GU, LDU, nU);
    const float g0 = pass_rows_out<BX>(w, twx, c.GU, LDU, nU, urp, P.dU_x + u_off, OutStart{c.sv, c.dv, c.xv});
    int par = 0;
    const double gamma0 = block_sum2f(g0, c.red, par);
    // CGNR
    double gamma = gamma0;
    bool conv = !(gamma0 > 1e-300);
    const double stop = (double)tol * (double)tol * gamma0;
    int it = 0;
    float bf = 0.f;                  // first direction: d = s
    for (; it < iters && !conv; ++it) {
        pass_rows_in<BX>(w, twx, c.GU, LDU, nU, urp, P.dU_x + u_off, ValNextDir{c.sv, c.dv, bf});
        __syncthreads();
        cols_times<BY, true>(c, twy, mx, c.GU, LDU, nU, c.GQ, mx, nQ);
        pass_rows_mask<BX>(w, twx, c.GQ, nQ, qmask);
        cols_times<BY, false>(c, twy, mx, c.GQ, mx, nQ, c.GU, LDU, nU);
        const float dw = pass_rows_out<BX>(w, twx, c.GU, LDU, nU, urp, P.dU_x + u_off, OutDot{c.wv, c.dv});
        const double delta = block_sum2f(dw, c.red, par);
        if (!(delta > 0)) break;
        const double alpha = gamma / delta;
        const float af = (float)alpha;
        float g2 = 0.f;
        for (int e = threadIdx.x; e < N; e += blockDim.x) {
            const float2 d = c.dv[e];
            float2 x = c.xv[e];
            x.x += af * d.x;
            x.y += af * d.y;
            c.xv[e] = x;
            const float2 sv = csub(c.sv[e], cscale(c.wv[e], af));
            c.sv[e] = sv;
            g2 += sv.x * sv.x + sv.y * sv.y;
        }
        const double gnew = block_sum2f(g2, c.red, par);
        bf = (float)(gnew / gamma);
        gamma = gnew;
        conv = gnew <= stop;
    }
    // corrected unknown spectrum into the tile's spectrum
    const int* Upup = P.dU_pup + u_off;
    const int* Uap = P.dU_ap + u_off;
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
        float sn, cs;
        sincosf(ph[Upup[e]], &sn, &cs);
        sp[Uap[e]] = cmul(c.xv[e], make_float2(cs, -sn));
    }
    __syncthreads();
    return conv ? it : -1 - it;
}

template <int B, int BN>
__global__ void __launch_bounds__(kDFThreads, 1)
k_darkfield_reg(DevPlan P, int n_tiles, const float* __restrict__ I, const float* __restrict__ phi,
                float2* __restrict__ spec, char* __restrict__ scratch, size_t per_block, int iters, float tol,
                int32_t* __restrict__ status, unsigned long long* __restrict__ counters, int* __restrict__ work) {
    constexpr int m = 16 * B, n = 16 * BN;
    constexpr int HWM = hw_area_m(B), HWN = HWSize<BN>::value;
    extern __shared__ float4 smem4[];
    char* sbase = reinterpret_cast<char*>(smem4);
    const DFRSmem SL = dfr_smem_layout(B, BN, P.band_u, P.band_q, P.max_N);
    DFCtx c;
    c.GU = reinterpret_cast<float2*>(sbase + SL.gu);
    float2* stage = reinterpret_cast<float2*>(sbase + SL.stage);
    c.dv = reinterpret_cast<float2*>(sbase + SL.c);
    c.sv = c.dv + P.max_N;
    c.wv = c.sv + P.max_N;
    float2* tw_m = c.wv + P.max_N;
    float2* tw_n = tw_m + 2 * m;
    c.tw_y = tw_n + 2 * n;
    c.tw_x = c.tw_y + 2 * m;
    c.red = reinterpret_cast<double*>(sbase + align16(SL.c + (size_t)3 * P.max_N * sizeof(float2) +
                                                      (size_t)2 * (m + n) * sizeof(float2) +
                                                      (size_t)4 * m * sizeof(float2)));
    c.tw_m = tw_m;

    make_step_twiddles(tw_m, P.tw_r, B);
    make_step_twiddles(tw_n, P.tw_n, BN);
    // TMEM for the known field: all 512 columns. One block of this kernel fills an SM's
    // register file (512 threads x 128 registers), so no other block of it holds TMEM
    // on the SM and the allocation does not wait (were there one, it would wait only
    // for that block's release at its end: blocks never wait on one another).
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5;
    if constexpr (uses_tmem(B)) {
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         :: "r"((uint32_t)__cvta_generic_to_shared(&tmem_base)), "r"(kTmemCols) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if constexpr (uses_tmem(B)) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        c.tm = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(kTmemSlotCols * (warp >> 2));
    } else {
        c.tm = 0;
    }

    HW wn;                           // image (n-grid) setup passes
    c.w.hw = wn.hw = threadIdx.x >> 4;
    c.w.t = wn.t = threadIdx.x & 15;
    c.w.mask = wn.mask = (threadIdx.x & 16) ? 0xFFFF0000u : 0x0000FFFFu;
    c.w.hs = reinterpret_cast<float2*>(sbase) + c.w.hw * HWM;
    wn.hs = reinterpret_cast<float2*>(sbase) + c.w.hw * HWN;

    c.xv = reinterpret_cast<float2*>(sbase + SL.x);
    char* base = scratch + (size_t)blockIdx.x * per_block;
    c.GQ = reinterpret_cast<float2*>(base);
    c.PF = c.GQ + (size_t)(P.band_q > P.band_p ? P.band_q : P.band_p) * m;   // column-major p, or F(I) rows
    c.bq = c.PF + (size_t)max(m * m, P.band_q * n);

    // tiles taken one at a time from the launch's counter (a block that meets skipped
    // background tiles goes on to the next, so uneven batches balance), or by stride
    __shared__ int s_next;
    auto take = [&](int prev) -> int {
        if (!work) return prev < 0 ? (int)blockIdx.x : prev + (int)gridDim.x;
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
            const int nQ = D.qy1 - D.qy0 + 1;
            const float* img = I + ((size_t)tile * P.n_img + D.led) * n * n;
            // b = F(I_j) on Q (setup transforms in the shared space of GU)
            pass_image_cols<BN>(wn, tw_n, stage, img, c.PF, D.qy0, nQ, D.tr != 0);
            pass_image_rows<BN>(wn, tw_n, c.PF, nQ, P.d_rowptr + D.qrp, P.dQ_x + D.q_off, c.bq);
            int r;
            if constexpr (B == 12) {     // the (row, column) grids the plan chooses from
                switch (16 * D.bx + D.by) {
                    case 16 * 12 + 6: r = df_solve<B, 12, 6>(c, P, D, sp, ph, iters, tol); break;
                    case 16 * 12 + 8: r = df_solve<B, 12, 8>(c, P, D, sp, ph, iters, tol); break;
                    case 16 * 12 + 9: r = df_solve<B, 12, 9>(c, P, D, sp, ph, iters, tol); break;
                    case 16 * 10 + 6: r = df_solve<B, 10, 6>(c, P, D, sp, ph, iters, tol); break;
                    case 16 * 10 + 8: r = df_solve<B, 10, 8>(c, P, D, sp, ph, iters, tol); break;
                    case 16 * 9 + 9: r = df_solve<B, 9, 9>(c, P, D, sp, ph, iters, tol); break;
                    default: r = df_solve<B, B, B>(c, P, D, sp, ph, iters, tol); break;
                }
            } else {
                r = df_solve<B, B, B>(c, P, D, sp, ph, iters, tol);
            }
            if (r < 0) notconv = true;
            if (threadIdx.x == 0 && counters) {
                atomicAdd(counters + 1, (unsigned long long)(r < 0 ? -1 - r : r));
                atomicAdd(counters + 2, 1ull);
                if (di < kCountedImages) atomicAdd(counters + 4 + di, (unsigned long long)(r < 0 ? -1 - r : r));
            }
        }
        if (threadIdx.x == 0 && notconv && status) atomicOr(status + tile, APIC_TILE_NOTCONV);
    }
    if constexpr (uses_tmem(B)) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (warp == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem_base), "r"(kTmemCols)
                         : "memory");
        }
    }
}

using DFRKernel = void (*)(DevPlan, int, const float*, const float*, float2*, char*, size_t, int, float, int32_t*,
                           unsigned long long*, int*);

DFRKernel dfr_kernel(int B, int BN) {
    if (B == 4 && BN == 4) return k_darkfield_reg<4, 4>;
    if (B == 6 && BN == 8) return k_darkfield_reg<6, 8>;
    if (B == 8 && BN == 8) return k_darkfield_reg<8, 8>;
    if (B == 12 && BN == 16) return k_darkfield_reg<12, 16>;
    if (B == 16 && BN == 16) return k_darkfield_reg<16, 16>;
    return nullptr;
}

int configure_dfr(int B, int BN, size_t smem) {
    DFRKernel f = dfr_kernel(B, BN);
    if (!f) return 0;
    if (raise_smem_limit((const void*)f, smem) != cudaSuccess)
        return 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kDFThreads, smem) != cudaSuccess) return 0;
    return occ;
}

cudaError_t launch_darkfield_reg(const DevPlan& P, int grid, size_t smem, int n_tiles, const float* I,
                                 const float* phi, float2* spec, void* scratch, size_t per_block, int iters,
                                 float tol, int32_t* status, unsigned long long* counters, int* work, cudaStream_t st) {
    DFRKernel f = dfr_kernel(P.mr / 16, P.h / 16);
    if (!f) return cudaErrorInvalidValue;
    if (work) {
        const cudaError_t e = cudaMemsetAsync(work, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    f<<<min(grid, n_tiles), kDFThreads, smem, st>>>(P, n_tiles, I, phi, spec, (char*)scratch, per_block, iters, tol,
                                                  status, counters, work);
    return cudaGetLastError();
}

}  // namespace apic
