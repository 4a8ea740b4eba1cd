// net.cu - the Zernike-predicting network: input features, BF16 tensor-core
// layers, training (loss, backward, AdamW) and the C interface apic_net_*.
//
// Input per tile: 8 channels f = log(|F(I)| / |F(I)(0)| + 1e-4) on the 64 x 64
// low-frequency crop (kx, ky in [-32, 32)) of each NA-matching image's
// intensity spectrum, plus the tile position (u, v). Layers, NHWC on the device:
//   conv3x3 8->32, ReLU, maxpool2 | conv 32->64, ReLU, pool | conv 64->128,
//   ReLU, pool | conv 128->256, ReLU, global mean | concat (u, v)
//   | dense 258->256, ReLU | dense 256->12 (Noll 4..15).
// Weights and the activations that feed a layer are BF16, products accumulate
// in FP32 on the tensor cores (mma.sync m16n8k16), gradients and the AdamW
// master weights are FP32. Every convolution (forward, data gradient, weight
// gradient) and dense layer is one generic GEMM kernel whose operands are
// gathered through loader functors (implicit im2col), with split-K and atomic
// accumulation for the weight gradients.
//
// Parameters: six matrices W_l [out_l][taps_l + 1] stored back to back in FP32,
// the bias in the last column; convolution taps are ordered (dy, dx, c_in),
// dense taps are the input features.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/apic.h"
#include "internal.cuh"
#include "regfft.cuh"

namespace apic {
namespace net {

constexpr int kCrop = 64;
constexpr int kIn = 8;
constexpr int kHidden = 256;
constexpr int kOut = 12;
constexpr int kC0 = 8, kC1 = 32, kC2 = 64, kC3 = 128, kC4 = 256;
constexpr int kHin = kC4 + 2;

// FP32 parameters W_l [rows][taps + 1] back to back (off, ld); the BF16 copy the
// GEMMs read has its rows padded to a multiple of 8 values (offp, ldp) so that
// 16-byte vector loads stay aligned.
struct Layout {
    size_t off[6], offp[6];
    int rows[6], taps[6];
    size_t total, total_pad;
    Layout() {
        const int r[6] = {kC1, kC2, kC3, kC4, kHidden, kOut};
        const int t[6] = {9 * kC0, 9 * kC1, 9 * kC2, 9 * kC3, kHin, kHidden};
        size_t o = 0, op = 0;
        for (int l = 0; l < 6; ++l) {
            off[l] = o;
            offp[l] = op;
            rows[l] = r[l];
            taps[l] = t[l];
            o += (size_t)r[l] * (t[l] + 1);
            op += (size_t)r[l] * ((t[l] + 1 + 7) / 8 * 8);
        }
        total = o;
        total_pad = op;
    }
    __host__ __device__ int ld(int l) const { return taps[l] + 1; }
    __host__ __device__ int ldp(int l) const { return (taps[l] + 1 + 7) / 8 * 8; }
    // index in the padded copy of flat parameter i
    __device__ size_t padded(size_t i) const {
        int l = 5;
        while (l > 0 && i < off[l]) --l;
        const size_t q = i - off[l];
        const size_t r = q / (size_t)ld(l), c = q - r * (size_t)ld(l);
        return offp[l] + r * (size_t)ldp(l) + c;
    }
};

// ------------------------------------------------------------------ features
// One block per (tile, image), persistent: forward transform of every row,
// keep the 64 columns kx in [-32, 32), forward transform of those columns,
// keep ky in [-32, 32), log of the magnitude relative to the DC term (the
// image sum). Output NHWC: feat[tile][ky + 32][kx + 32][image].
template <int BN>
__global__ void __launch_bounds__(512, 1) k_features(DevPlan P, int n_tiles, const float* __restrict__ I,
                                                     float* __restrict__ feat, float2* __restrict__ scratch) {
    constexpr int n = 16 * BN, HWS = HWSize<BN>::value, NHW = 32, S = Slots<BN>::value;
    extern __shared__ float4 smem4[];
    float2* hw_area = reinterpret_cast<float2*>(smem4);
    float2* tw = hw_area + NHW * HWS;
    __shared__ double red[32];
    make_step_twiddles(tw, P.tw_n, BN);
    __syncthreads();
    const int hw = threadIdx.x >> 4, t = threadIdx.x & 15;
    const HalfWarp h{t, (threadIdx.x & 16) ? 0xFFFF0000u : 0x0000FFFFu, hw_area + hw * HWS};
    float2* G = scratch + (size_t)blockIdx.x * n * kCrop;   // [row][kept column]
    const int nprob = n_tiles * kIn;
    for (int prob = blockIdx.x; prob < nprob; prob += gridDim.x) {
        const int tile = prob / kIn, i = prob - tile * kIn;
        const float* img = I + ((size_t)tile * P.n_img + i) * n * n;
        double s = 0;
        const float4* img4 = reinterpret_cast<const float4*>(img);
        for (int q = threadIdx.x; q < n * n / 4; q += blockDim.x) {
            const float4 v = img4[q];
            s += (double)v.x + v.y + v.z + v.w;
        }
        s = block_sum(s, red);
        const float inv_dc = s > 0 ? (float)(1.0 / s) : 0.f;
        for (int r = hw; r < n; r += NHW) {
            float2 v[BN], o[S][16];
#pragma unroll
            for (int j = 0; j < BN; ++j) v[j] = make_float2(img[(size_t)r * n + t + 16 * j], 0.f);
            fft_a<BN, false>(v, o, h, tw);
#pragma unroll
            for (int sl = 0; sl < S; ++sl)
                if (t + 16 * sl < BN) {
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) {
                        const int kx = t + 16 * sl + BN * k1;
                        const int sx = kx < n / 2 ? kx : kx - n;
                        if (sx >= -kCrop / 2 && sx < kCrop / 2) G[(size_t)r * kCrop + sx + kCrop / 2] = o[sl][k1];
                    }
                }
        }
        __syncthreads();
        float* f = feat + (size_t)tile * kCrop * kCrop * kIn + i;
        for (int c = hw; c < kCrop; c += NHW) {
            float2 v[BN], o[S][16];
#pragma unroll
            for (int j = 0; j < BN; ++j) v[j] = G[(size_t)(t + 16 * j) * kCrop + c];
            fft_a<BN, false>(v, o, h, tw);
#pragma unroll
            for (int sl = 0; sl < S; ++sl)
                if (t + 16 * sl < BN) {
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) {
                        const int ky = t + 16 * sl + BN * k1;
                        const int sy = ky < n / 2 ? ky : ky - n;
                        if (sy >= -kCrop / 2 && sy < kCrop / 2)
                            f[((size_t)(sy + kCrop / 2) * kCrop + c) * kIn] =
                                logf(sqrtf(cabs2(o[sl][k1])) * inv_dc + 1e-4f);
                    }
                }
        }
        __syncthreads();
    }
}

size_t features_smem(int BN) {
    return (size_t)32 * std::max(17 * BN, 16 * (BN + 1)) * sizeof(float2) + (size_t)2 * 16 * BN * sizeof(float2);
}

// ------------------------------------------------------------------ GEMM
// C(m, n) = sum_k A(m, k) B(k, n): bf16 operands, fp32 accumulation.
// Block tile 64 x 64 x 32, four warps of 32 x 32; blockIdx.z splits K (the
// epilogue must then accumulate atomically).
constexpr int kBM = 64, kBN = 64, kBK = 32, kLD = kBK + 8;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Staging of 16 consecutive k of one A row (m fixed) or one B column (n fixed)
// into 16 BF16 values of shared memory (16-byte aligned). Loaders whose data is
// contiguous along k provide segA / segB with vector loads; the others go
// through their element loaders.
template <class F, class = void>
struct HasSegA : std::false_type {};
template <class F>
struct HasSegA<F, std::void_t<decltype(std::declval<const F&>().segA(0, 0, 0, (__nv_bfloat16*)nullptr))>>
    : std::true_type {};
template <class F, class = void>
struct HasSegB : std::false_type {};
template <class F>
struct HasSegB<F, std::void_t<decltype(std::declval<const F&>().segB(0, 0, 0, (__nv_bfloat16*)nullptr))>>
    : std::true_type {};

__device__ __forceinline__ void zero16(__nv_bfloat16* dst) {
    reinterpret_cast<uint4*>(dst)[0] = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4*>(dst)[1] = make_uint4(0, 0, 0, 0);
}

__device__ __forceinline__ unsigned pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const unsigned*>(&h);
}

// 8 floats (two float4, 16-byte aligned source) -> 8 BF16 (one uint4)
__device__ __forceinline__ uint4 f8_to_bf16(const float* src) {
    const float4 a = reinterpret_cast<const float4*>(src)[0], b = reinterpret_cast<const float4*>(src)[1];
    return make_uint4(pack_bf16(a.x, a.y), pack_bf16(a.z, a.w), pack_bf16(b.x, b.y), pack_bf16(b.z, b.w));
}

template <class F>
__device__ __forceinline__ void stage_a(const F& f, bool valid, int m, int k0, int kend, __nv_bfloat16* dst) {
    if (!valid) {
        zero16(dst);
    } else if constexpr (HasSegA<F>::value) {
        f.segA(m, k0, kend, dst);
    } else {
#pragma unroll 4
        for (int c = 0; c < 16; ++c) dst[c] = __float2bfloat16(k0 + c < kend ? f(m, k0 + c) : 0.f);
    }
}

template <class F>
__device__ __forceinline__ void stage_b(const F& f, bool valid, int n, int k0, int kend, __nv_bfloat16* dst) {
    if (!valid) {
        zero16(dst);
    } else if constexpr (HasSegB<F>::value) {
        f.segB(k0, kend, n, dst);
    } else {
#pragma unroll 4
        for (int c = 0; c < 16; ++c) dst[c] = __float2bfloat16(k0 + c < kend ? f(k0 + c, n) : 0.f);
    }
}

template <class LA, class LB, class EP>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, int k_split, LA la, LB lb, EP ep) {
    __shared__ __align__(16) __nv_bfloat16 As[kBM * kLD];
    __shared__ __align__(16) __nv_bfloat16 Bs[kBN * kLD];
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int kb = blockIdx.z * k_split, ke = min(K, kb + k_split);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, tg = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    // staging: thread -> (row sr of the tile, 16 consecutive k from sc)
    const int sr = threadIdx.x >> 1, sc = (threadIdx.x & 1) * 16;
    const int am = m0 + sr, bn = n0 + sr;
    for (int k0 = kb; k0 < ke; k0 += kBK) {
        stage_a(la, am < M, am, k0 + sc, ke, As + sr * kLD + sc);
        stage_b(lb, bn < N, bn, k0 + sc, ke, Bs + sr * kLD + sc);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            unsigned a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const __nv_bfloat16* p = As + (wm + i * 16 + g) * kLD + kk + tg * 2;
                a[i][0] = *reinterpret_cast<const unsigned*>(p);
                a[i][1] = *reinterpret_cast<const unsigned*>(p + 8 * kLD);
                a[i][2] = *reinterpret_cast<const unsigned*>(p + 8);
                a[i][3] = *reinterpret_cast<const unsigned*>(p + 8 * kLD + 8);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const __nv_bfloat16* p = Bs + (wn + j * 8 + g) * kLD + kk + tg * 2;
                b[j][0] = *reinterpret_cast<const unsigned*>(p);
                b[j][1] = *reinterpret_cast<const unsigned*>(p + 8);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + i * 16 + g + (e >= 2 ? 8 : 0);
                const int nn = n0 + wn + j * 8 + tg * 2 + (e & 1);
                if (m < M && nn < N) ep(m, nn, acc[i][j][e]);
            }
}

// splits > 1 only with an accumulating epilogue.
template <class LA, class LB, class EP>
cudaError_t gemm(int M, int N, int K, int splits, LA la, LB lb, EP ep, cudaStream_t st, long long* launches) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    splits = std::max(1, std::min(splits, (K + kBK - 1) / kBK));
    int k_split = (K + splits - 1) / splits;
    k_split = (k_split + kBK - 1) / kBK * kBK;
    splits = (K + k_split - 1) / k_split;
    const dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, splits);
    k_gemm<<<grid, 128, 0, st>>>(M, N, K, k_split, la, lb, ep);
    if (launches) ++*launches;
    return cudaGetLastError();
}

// ---- operand loaders (A(m, k) or B(k, n), returning float)
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// im2col of an NHWC H x H map with C channels for a 3x3, pad-1 convolution:
// (m, k) with m = (b, y, x) and k = (dy, dx, c); k = 9 C is the bias column.
// Serves as A of the forward pass and, called as (pixel, tap), as B of the
// weight gradient.
template <int H, int C, class T>
struct ConvIn {
    const T* x;
    __device__ float operator()(int m, int k) const {
        if (k >= 9 * C) return 1.f;
        const int c = k % C, s = k / C, dy = s / 3, dx = s - 3 * dy;
        const int q = m / H, xx = m - q * H + dx - 1;
        const int b = q / H, yy = q - b * H + dy - 1;
        if ((unsigned)yy >= (unsigned)H || (unsigned)xx >= (unsigned)H) return 0.f;
        return to_f(x[(((size_t)b * H + yy) * H + xx) * C + c]);
    }
    // address of channel c of tap s at output pixel m, or NULL in the padding
    __device__ const T* tap(int m, int s, int c) const {
        const int dy = s / 3, dx = s - 3 * dy;
        const int q = m / H, xx = m - q * H + dx - 1;
        const int b = q / H, yy = q - b * H + dy - 1;
        if ((unsigned)yy >= (unsigned)H || (unsigned)xx >= (unsigned)H) return nullptr;
        return x + (((size_t)b * H + yy) * H + xx) * C + c;
    }
    // 16 consecutive taps of a row: one tap's 16 channels (C % 16 == 0, BF16
    // maps) or two taps' 8 channels (C == 8, FP32 input); vector loads
    __device__ void segA(int m, int k0, int kend, __nv_bfloat16* dst) const {
        if (k0 + 16 <= kend && k0 + 16 <= 9 * C) {
            if constexpr (std::is_same<T, __nv_bfloat16>::value && C % 16 == 0) {
                const int s = k0 / C;
                const T* p = tap(m, s, k0 - s * C);
                if (p) {
                    reinterpret_cast<uint4*>(dst)[0] = reinterpret_cast<const uint4*>(p)[0];
                    reinterpret_cast<uint4*>(dst)[1] = reinterpret_cast<const uint4*>(p)[1];
                } else {
                    zero16(dst);
                }
                return;
            } else if constexpr (std::is_same<T, float>::value && C == 8) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const T* p = tap(m, k0 / 8 + h, 0);
                    reinterpret_cast<uint4*>(dst)[h] = p ? f8_to_bf16(p) : make_uint4(0, 0, 0, 0);
                }
                return;
            }
        }
#pragma unroll 4
        for (int c = 0; c < 16; ++c) dst[c] = __float2bfloat16(k0 + c < kend ? (*this)(m, k0 + c) : 0.f);
    }
};
// (co, pixel) of the pre-activation gradient dz = dr * [r > 0]
template <int C>
struct ReluGradT {
    const float* g;
    const __nv_bfloat16* r;
    __device__ float operator()(int c, int m) const {
        const size_t i = (size_t)m * C + c;
        return __bfloat162float(r[i]) > 0.f ? g[i] : 0.f;
    }
};
// data gradient of the convolution: (m, k) with m = (b, y, x) of the input map
// and k = (dy, dx, co) reads dz at (y - dy + 1, x - dx + 1)
template <int H, int Co>
struct DzShift {
    const float* g;
    const __nv_bfloat16* r;
    __device__ float operator()(int m, int k) const {
        const int co = k % Co, s = k / Co, dy = s / 3, dx = s - 3 * dy;
        const int q = m / H, xx = m - q * H - dx + 1;
        const int b = q / H, yy = q - b * H - dy + 1;
        if ((unsigned)yy >= (unsigned)H || (unsigned)xx >= (unsigned)H) return 0.f;
        const size_t i = (((size_t)b * H + yy) * H + xx) * Co + co;
        return __bfloat162float(r[i]) > 0.f ? g[i] : 0.f;
    }
    // 16 consecutive output channels of one tap (Co % 16 == 0): vector loads of
    // the gradient and of the activation that masks it
    __device__ void segA(int m, int k0, int kend, __nv_bfloat16* dst) const {
        static_assert(Co % 16 == 0, "16 channels per segment");
        if (k0 + 16 <= kend) {
            const int s = k0 / Co, co = k0 - s * Co, dy = s / 3, dx = s - 3 * dy;
            const int q = m / H, xx = m - q * H - dx + 1;
            const int b = q / H, yy = q - b * H - dy + 1;
            if ((unsigned)yy >= (unsigned)H || (unsigned)xx >= (unsigned)H) {
                zero16(dst);
                return;
            }
            const size_t i = (((size_t)b * H + yy) * H + xx) * Co + co;
            const float4* g4 = reinterpret_cast<const float4*>(g + i);
            const uint4* r4 = reinterpret_cast<const uint4*>(r + i);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint4 rv = r4[h];
                const __nv_bfloat16* rb = reinterpret_cast<const __nv_bfloat16*>(&rv);
                const float4 a = g4[2 * h], c = g4[2 * h + 1];
                const float v[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
                unsigned w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    w[e] = pack_bf16(__bfloat162float(rb[2 * e]) > 0.f ? v[2 * e] : 0.f,
                                     __bfloat162float(rb[2 * e + 1]) > 0.f ? v[2 * e + 1] : 0.f);
                reinterpret_cast<uint4*>(dst)[h] = make_uint4(w[0], w[1], w[2], w[3]);
            }
            return;
        }
#pragma unroll 4
        for (int c = 0; c < 16; ++c) dst[c] = __float2bfloat16(k0 + c < kend ? (*this)(m, k0 + c) : 0.f);
    }
};
// (k = (dy, dx, co), n = ci) -> W[co][(dy, dx, ci)]
template <int Ci, int Co>
struct WFlip {
    const __nv_bfloat16* w;
    int ld;
    __device__ float operator()(int k, int n) const {
        const int co = k % Co, s = k / Co;
        return __bfloat162float(w[(size_t)co * ld + s * Ci + n]);
    }
};
struct WT {                 // B(k, n) = W[n][k]; rows padded to multiples of 8
    const __nv_bfloat16* w;
    int ld;
    __device__ float operator()(int k, int n) const { return __bfloat162float(w[(size_t)n * ld + k]); }
    __device__ void segB(int k0, int kend, int n, __nv_bfloat16* dst) const {
        const __nv_bfloat16* p = w + (size_t)n * ld + k0;
        if (k0 + 16 <= kend) {
            reinterpret_cast<uint4*>(dst)[0] = reinterpret_cast<const uint4*>(p)[0];
            reinterpret_cast<uint4*>(dst)[1] = reinterpret_cast<const uint4*>(p)[1];
            return;
        }
#pragma unroll 4
        for (int c = 0; c < 16; ++c) dst[c] = k0 + c < kend ? p[c] : __float2bfloat16(0.f);
    }
};
struct WN {                 // B(k, n) = W[k][n]
    const __nv_bfloat16* w;
    int ld;
    __device__ float operator()(int k, int n) const { return __bfloat162float(w[(size_t)k * ld + n]); }
};
struct Mat {                // (r, c) -> p[r][c]
    const float* p;
    int ld;
    __device__ float operator()(int r, int c) const { return p[(size_t)r * ld + c]; }
    __device__ void segA(int r, int k0, int kend, __nv_bfloat16* dst) const {
        const float* q = p + (size_t)r * ld + k0;
        if (k0 + 16 <= kend && (ld & 3) == 0) {
            reinterpret_cast<uint4*>(dst)[0] = f8_to_bf16(q);
            reinterpret_cast<uint4*>(dst)[1] = f8_to_bf16(q + 8);
            return;
        }
#pragma unroll 4
        for (int c = 0; c < 16; ++c) dst[c] = __float2bfloat16(k0 + c < kend ? q[c] : 0.f);
    }
};
struct MatT {               // (r, c) -> p[c][r]
    const float* p;
    int ld;
    __device__ float operator()(int r, int c) const { return p[(size_t)c * ld + r]; }
};
struct MatBias {            // (r, c) -> p[r][c], 1 in column `cols` (bias column)
    const float* p;
    int ld, cols;
    __device__ float operator()(int r, int c) const { return c >= cols ? 1.f : p[(size_t)r * ld + c]; }
};

// ---- epilogues
struct EpConv {             // r = relu(acc + bias) as bf16, [m][ld]
    __nv_bfloat16* out;
    const float* bias;
    int bias_stride, ld;
    __device__ void operator()(int m, int n, float v) const {
        out[(size_t)m * ld + n] = __float2bfloat16(fmaxf(v + bias[(size_t)n * bias_stride], 0.f));
    }
};
struct EpDense {            // fp32 acc + bias, optional ReLU
    float* out;
    const float* bias;
    int bias_stride, ld;
    bool relu;
    __device__ void operator()(int m, int n, float v) const {
        const float r = v + bias[(size_t)n * bias_stride];
        out[(size_t)m * ld + n] = relu ? fmaxf(r, 0.f) : r;
    }
};
struct EpStore {
    float* out;
    int ld;
    __device__ void operator()(int m, int n, float v) const { out[(size_t)m * ld + n] = v; }
};
struct EpAtomic {
    float* out;
    int ld;
    __device__ void operator()(int m, int n, float v) const { atomicAdd(out + (size_t)m * ld + n, v); }
};

// ------------------------------------------------------------------ other layers
// 2 x 2 max-pool of an NHWC bf16 map (first maximum in (dy, dx) order), with the
// chosen position kept for the backward pass.
__global__ void k_maxpool(const __nv_bfloat16* __restrict__ r, __nv_bfloat16* __restrict__ out,
                          uint8_t* __restrict__ arg, int B, int H, int C) {
    const int Ho = H / 2;
    const size_t total = (size_t)B * Ho * Ho * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int x = (int)(q % Ho), y = (int)((q / Ho) % Ho), b = (int)(q / ((size_t)Ho * Ho));
        float best = -INFINITY;
        int bi = 0;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float v = __bfloat162float(r[(((size_t)b * H + 2 * y + (s >> 1)) * H + 2 * x + (s & 1)) * C + c]);
            if (v > best) {
                best = v;
                bi = s;
            }
        }
        out[i] = __float2bfloat16(best);
        arg[i] = (uint8_t)bi;
    }
}

__global__ void k_maxpool_back(const float* __restrict__ g, const uint8_t* __restrict__ arg, float* __restrict__ gin,
                               int B, int H, int C) {
    const int Ho = H / 2;
    const size_t total = (size_t)B * Ho * Ho * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int x = (int)(q % Ho), y = (int)((q / Ho) % Ho), b = (int)(q / ((size_t)Ho * Ho));
        const int a = arg[i];
#pragma unroll
        for (int s = 0; s < 4; ++s)
            gin[(((size_t)b * H + 2 * y + (s >> 1)) * H + 2 * x + (s & 1)) * C + c] = s == a ? g[i] : 0.f;
    }
}

// global mean over the HW pixels of the last ReLU map, then (u, v)
__global__ void k_gap_concat(const __nv_bfloat16* __restrict__ r, const float* __restrict__ uv,
                             float* __restrict__ hin, int HW, int C) {
    const int b = blockIdx.x;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float s = 0.f;
        for (int p = 0; p < HW; ++p) s += __bfloat162float(r[((size_t)b * HW + p) * C + c]);
        hin[(size_t)b * (C + 2) + c] = s / (float)HW;
    }
    if (threadIdx.x < 2) hin[(size_t)b * (C + 2) + C + threadIdx.x] = uv ? uv[2 * b + threadIdx.x] : 0.f;
}

__global__ void k_gap_back(const float* __restrict__ ghin, float* __restrict__ gr, int B, int HW, int C) {
    const size_t total = (size_t)B * HW * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const int b = (int)(i / ((size_t)HW * C));
        gr[i] = ghin[(size_t)b * (C + 2) + c] / (float)HW;
    }
}

// mean squared error over the batch and the 12 outputs (Noll 4..15 of the
// [b][15] targets) and its gradient
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ target, float* __restrict__ gy,
                       float* __restrict__ loss, int B) {
    __shared__ double red[32];
    double acc = 0;
    for (int i = threadIdx.x; i < B * kOut; i += blockDim.x) {
        const int b = i / kOut, j = i - b * kOut;
        const float d = y[i] - target[(size_t)b * APIC_N_ZERNIKE + 3 + j];
        gy[i] = 2.f * d / (float)(B * kOut);
        acc += (double)d * d;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0 && loss) *loss = (float)(acc / (B * kOut));
}

__global__ void k_pack_out(const float* __restrict__ y, float* __restrict__ out, int B) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * APIC_N_ZERNIKE; i += gridDim.x * blockDim.x) {
        const int b = i / APIC_N_ZERNIKE, j = i - b * APIC_N_ZERNIKE;
        out[i] = j < 3 ? 0.f : y[(size_t)b * kOut + j - 3];
    }
}

__global__ void k_relu_mask(float* __restrict__ g, const float* __restrict__ h, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(h[i] > 0.f)) g[i] = 0.f;
}

__global__ void k_cast_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t n, Layout L) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[L.padded(i)] = __float2bfloat16(src[i]);
}

// AdamW with bias-corrected moments and decoupled weight decay; refreshes the bf16 copy.
__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, __nv_bfloat16* __restrict__ pbf, size_t n, float lr, float b1, float b2,
                        float eps, float wd, float c1, float c2, Layout L) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
        p[i] = pi;
        pbf[L.padded(i)] = __float2bfloat16(pi);
    }
}

int blocks_for(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 4096)); }

}  // namespace net

// Features of n_tiles tiles (the first 8 images of each stack) with the plan's
// register transforms; `scratch` holds h * 64 complex values per block.
cudaError_t launch_features(const DevPlan& P, int grid, int n_tiles, const float* I, float* feat, float2* scratch,
                            cudaStream_t st) {
    using namespace net;
    const int BN = P.h / 16;
    const size_t smem = features_smem(BN);
    grid = std::min(grid, n_tiles * kIn);
    if (grid < 1) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    switch (BN) {
        case 4:
            e = raise_smem_limit((const void*)k_features<4>, smem);
            if (e == cudaSuccess) k_features<4><<<grid, 512, smem, st>>>(P, n_tiles, I, feat, scratch);
            break;
        case 8:
            e = raise_smem_limit((const void*)k_features<8>, smem);
            if (e == cudaSuccess) k_features<8><<<grid, 512, smem, st>>>(P, n_tiles, I, feat, scratch);
            break;
        case 16:
            e = raise_smem_limit((const void*)k_features<16>, smem);
            if (e == cudaSuccess) k_features<16><<<grid, 512, smem, st>>>(P, n_tiles, I, feat, scratch);
            break;
        case 32:
            e = raise_smem_limit((const void*)k_features<32>, smem);
            if (e == cudaSuccess) k_features<32><<<grid, 512, smem, st>>>(P, n_tiles, I, feat, scratch);
            break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

size_t feature_floats() { return (size_t)net::kCrop * net::kCrop * net::kIn; }

}  // namespace apic

using namespace apic;
using namespace apic::net;

struct apic_net {
    int max_batch = 0;
    Layout L;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16* wbf = nullptr;            // bf16 copy of the parameters
    // forward state of the last apic_net_forward
    const float* in = nullptr;               // caller's features
    int last_batch = 0;
    __nv_bfloat16 *r[4] = {}, *pool[3] = {};
    uint8_t* arg[3] = {};
    float *hin = nullptr, *h4 = nullptr, *y = nullptr;
    // gradients of activations
    float *g_r[4] = {}, *g_pool[3] = {}, *g_hin = nullptr, *g_h4 = nullptr, *g_y = nullptr;
    long long launches = 0;
    std::vector<void*> allocs;
};

namespace {

apic_status net_fail(apic_status s, const std::string& m) {
    record_error((int)s, m.c_str());
    return s;
}

#define NET_TRY(expr)                                                                                         \
    do {                                                                                                      \
        cudaError_t _e = (expr);                                                                              \
        if (_e != cudaSuccess) return net_fail(APIC_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

template <typename T>
bool nalloc(apic_net* n, T** p, size_t count) {
    if (cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    n->allocs.push_back((void*)*p);
    return true;
}

// split-K factor of a weight-gradient GEMM: ~256 pixels per block, so even the small
// late layers spread over a few thousand blocks
int split_for(long long K) { return (int)std::max(1LL, std::min(512LL, K / 256)); }

}  // namespace

namespace apic {

// Forward pass on `B` tiles; out15 [B][15] (Noll 1..3 zero) may be NULL.
cudaError_t net_predict(apic_net* n, int B, const float* feat, const float* uv, float* out15, cudaStream_t st) {
    const Layout& L = n->L;
    long long* nl = &n->launches;
    n->in = feat;
    n->last_batch = B;
    cudaError_t e;
#define NET_STEP(x)                          \
    if ((e = (x)) != cudaSuccess) return e;
#define NET_POOL(l, H, C)                                                                                        \
    k_maxpool<<<blocks_for((size_t)B * (H / 2) * (H / 2) * C), 256, 0, st>>>(n->r[l], n->pool[l], n->arg[l], B, H, \
                                                                           C);                                    \
    ++*nl;                                                                                                       \
    NET_STEP(cudaGetLastError());
    NET_STEP(gemm(B * 64 * 64, kC1, 9 * kC0, 1, ConvIn<64, kC0, float>{feat}, WT{n->wbf + L.offp[0], L.ldp(0)},
                  EpConv{n->r[0], n->params + L.off[0] + L.taps[0], L.ld(0), kC1}, st, nl));
    NET_POOL(0, 64, kC1);
    NET_STEP(gemm(B * 32 * 32, kC2, 9 * kC1, 1, ConvIn<32, kC1, __nv_bfloat16>{n->pool[0]},
                  WT{n->wbf + L.offp[1], L.ldp(1)}, EpConv{n->r[1], n->params + L.off[1] + L.taps[1], L.ld(1), kC2}, st,
                  nl));
    NET_POOL(1, 32, kC2);
    NET_STEP(gemm(B * 16 * 16, kC3, 9 * kC2, 1, ConvIn<16, kC2, __nv_bfloat16>{n->pool[1]},
                  WT{n->wbf + L.offp[2], L.ldp(2)}, EpConv{n->r[2], n->params + L.off[2] + L.taps[2], L.ld(2), kC3}, st,
                  nl));
    NET_POOL(2, 16, kC3);
    NET_STEP(gemm(B * 8 * 8, kC4, 9 * kC3, 1, ConvIn<8, kC3, __nv_bfloat16>{n->pool[2]},
                  WT{n->wbf + L.offp[3], L.ldp(3)}, EpConv{n->r[3], n->params + L.off[3] + L.taps[3], L.ld(3), kC4}, st,
                  nl));
    k_gap_concat<<<B, 256, 0, st>>>(n->r[3], uv, n->hin, 64, kC4);
    ++*nl;
    NET_STEP(cudaGetLastError());
    NET_STEP(gemm(B, kHidden, kHin, 1, Mat{n->hin, kHin}, WT{n->wbf + L.offp[4], L.ldp(4)},
                  EpDense{n->h4, n->params + L.off[4] + L.taps[4], L.ld(4), kHidden, true}, st, nl));
    NET_STEP(gemm(B, kOut, kHidden, 1, Mat{n->h4, kHidden}, WT{n->wbf + L.offp[5], L.ldp(5)},
                  EpDense{n->y, n->params + L.off[5] + L.taps[5], L.ld(5), kOut, false}, st, nl));
    if (out15) {
        k_pack_out<<<(B * APIC_N_ZERNIKE + 255) / 256, 256, 0, st>>>(n->y, out15, B);
        ++*nl;
        NET_STEP(cudaGetLastError());
    }
#undef NET_POOL
#undef NET_STEP
    return cudaSuccess;
}

int net_max_batch(const apic_net* n) { return n->max_batch; }
long long net_launches(const apic_net* n) { return n->launches; }

}  // namespace apic

extern "C" {

size_t apic_net_param_count(void) { return Layout().total; }

size_t apic_net_feature_count(void) { return feature_floats(); }

apic_status apic_net_create(int max_batch, apic_net** out) {
    if (!out) return net_fail(APIC_EINVAL, "NULL output handle");
    *out = nullptr;
    if (max_batch < 1 || max_batch > 65536) return net_fail(APIC_EINVAL, "max_batch must be in [1, 65536]");
    apic_net* n = new apic_net();
    n->max_batch = max_batch;
    const size_t P = n->L.total, B = (size_t)max_batch;
    bool ok = nalloc(n, &n->params, P) && nalloc(n, &n->grads, P) && nalloc(n, &n->m, P) && nalloc(n, &n->v, P) &&
              nalloc(n, &n->wbf, n->L.total_pad);
    const int C[4] = {kC1, kC2, kC3, kC4};
    int H = kCrop;
    for (int l = 0; l < 4 && ok; ++l) {
        ok = nalloc(n, &n->r[l], B * H * H * C[l]) && nalloc(n, &n->g_r[l], B * H * H * C[l]);
        if (ok && l < 3) {
            H /= 2;
            ok = nalloc(n, &n->pool[l], B * H * H * C[l]) && nalloc(n, &n->arg[l], B * H * H * C[l]) &&
                 nalloc(n, &n->g_pool[l], B * H * H * C[l]);
        }
    }
    ok = ok && nalloc(n, &n->hin, B * kHin) && nalloc(n, &n->g_hin, B * kHin) && nalloc(n, &n->h4, B * kHidden) &&
         nalloc(n, &n->g_h4, B * kHidden) && nalloc(n, &n->y, B * kOut) && nalloc(n, &n->g_y, B * kOut);
    if (!ok) {
        apic_net_destroy(n);
        return net_fail(APIC_ENOMEM, "network workspace allocation failed");
    }
    if (cudaMemset(n->params, 0, P * 4) != cudaSuccess || cudaMemset(n->grads, 0, P * 4) != cudaSuccess ||
        cudaMemset(n->m, 0, P * 4) != cudaSuccess || cudaMemset(n->v, 0, P * 4) != cudaSuccess ||
        cudaMemset(n->wbf, 0, n->L.total_pad * 2) != cudaSuccess) {
        cudaGetLastError();
        apic_net_destroy(n);
        return net_fail(APIC_ECUDA, "network initialisation failed");
    }
    *out = n;
    return APIC_OK;
}

apic_status apic_net_destroy(apic_net* n) {
    if (!n) return APIC_OK;
    cudaDeviceSynchronize();
    for (void* p : n->allocs) cudaFree(p);
    delete n;
    return APIC_OK;
}

apic_status apic_net_set_params(apic_net* n, const float* h, size_t count) {
    if (!n || !h || count != n->L.total) return net_fail(APIC_EINVAL, "expected apic_net_param_count() floats");
    NET_TRY(cudaDeviceSynchronize());
    NET_TRY(cudaMemcpy(n->params, h, count * 4, cudaMemcpyHostToDevice));
    k_cast_bf16<<<blocks_for(count), 256>>>(n->params, n->wbf, count, n->L);
    NET_TRY(cudaGetLastError());
    NET_TRY(cudaMemset(n->m, 0, count * 4));
    NET_TRY(cudaMemset(n->v, 0, count * 4));
    NET_TRY(cudaDeviceSynchronize());
    return APIC_OK;
}

// Value of key `key` in a flat JSON object: the string after it ("...") or the
// digits of a number; empty when absent. Enough for the checkpoint header, whose
// writer emits plain keys, strings and integers.
static std::string json_value(const std::string& js, const std::string& key) {
    const std::string k = "\"" + key + "\"";
    size_t p = js.find(k);
    if (p == std::string::npos) return "";
    p += k.size();
    while (p < js.size() && (js[p] == ' ' || js[p] == ':' || js[p] == '\t' || js[p] == '\n')) ++p;
    if (p >= js.size()) return "";
    if (js[p] == '"') {
        const size_t e = js.find('"', p + 1);
        return e == std::string::npos ? "" : js.substr(p + 1, e - p - 1);
    }
    size_t e = p;
    while (e < js.size() && js[e] >= '0' && js[e] <= '9') ++e;
    return js.substr(p, e - p);
}

apic_status apic_net_load(apic_net* n, const void* blob, size_t bytes) {
    static const char kMagic[8] = {'A', 'P', 'I', 'C', 'N', 'B', '1', '6'};
    if (!blob) return net_fail(APIC_EINVAL, "NULL blob");
    const unsigned char* b = static_cast<const unsigned char*>(blob);
    if (bytes < 12 || std::memcmp(b, kMagic, 8) != 0) return net_fail(APIC_EINVAL, "not an APICNB16 checkpoint");
    const size_t L = (size_t)b[8] | ((size_t)b[9] << 8) | ((size_t)b[10] << 16) | ((size_t)b[11] << 24);
    if (L > bytes - 12) return net_fail(APIC_EINVAL, "checkpoint header runs past the blob");
    const std::string head(reinterpret_cast<const char*>(b + 12), L);
    if (json_value(head, "format") != "apic-net-bf16") return net_fail(APIC_EINVAL, "checkpoint format is not apic-net-bf16");
    const std::string cs = json_value(head, "count");
    const Layout lay;
    if (cs.empty() || cs.size() > 12 || std::stoull(cs) != (unsigned long long)lay.total)
        return net_fail(APIC_EINVAL, "checkpoint count differs from apic_net_param_count()");
    if (bytes != 12 + L + 2 * lay.total) return net_fail(APIC_EINVAL, "checkpoint size does not match its count");
    if (!n) return APIC_OK;                          // validation only
    std::vector<float> v(lay.total);
    const unsigned char* q = b + 12 + L;
    for (size_t i = 0; i < lay.total; ++i) {
        const uint32_t bits = ((uint32_t)q[2 * i] | ((uint32_t)q[2 * i + 1] << 8)) << 16;
        std::memcpy(&v[i], &bits, 4);
    }
    return apic_net_set_params(n, v.data(), v.size());
}

apic_status apic_net_get_params(const apic_net* n, float* h, size_t count) {
    if (!n || !h || count != n->L.total) return net_fail(APIC_EINVAL, "expected apic_net_param_count() floats");
    NET_TRY(cudaDeviceSynchronize());
    NET_TRY(cudaMemcpy(h, n->params, count * 4, cudaMemcpyDeviceToHost));
    return APIC_OK;
}

apic_status apic_net_get_grads(const apic_net* n, float* h, size_t count) {
    if (!n || !h || count != n->L.total) return net_fail(APIC_EINVAL, "expected apic_net_param_count() floats");
    NET_TRY(cudaDeviceSynchronize());
    NET_TRY(cudaMemcpy(h, n->grads, count * 4, cudaMemcpyDeviceToHost));
    return APIC_OK;
}

apic_status apic_net_forward(apic_net* n, int batch, const float* feat, const float* uv, float* out15,
                             void* stream) {
    if (!n || !feat) return net_fail(APIC_EINVAL, "NULL network or features");
    if (batch < 1 || batch > n->max_batch) return net_fail(APIC_EINVAL, "batch must be in [1, max_batch]");
    if (reinterpret_cast<uintptr_t>(feat) & 15) return net_fail(APIC_EINVAL, "features must be 16-byte aligned");
    NET_TRY(net_predict(n, batch, feat, uv, out15, (cudaStream_t)stream));
    return APIC_OK;
}

apic_status apic_net_backward(apic_net* n, const float* target15, float* loss, void* stream) {
    if (!n || !target15) return net_fail(APIC_EINVAL, "NULL network or target");
    if (n->last_batch < 1) return net_fail(APIC_EINVAL, "backward needs a preceding forward");
    cudaStream_t st = (cudaStream_t)stream;
    const int B = n->last_batch;
    const Layout& L = n->L;
    long long* nl = &n->launches;
    NET_TRY(cudaMemsetAsync(n->grads, 0, L.total * sizeof(float), st));
    k_loss<<<1, 256, 0, st>>>(n->y, target15, n->g_y, loss, B);
    ++*nl;
    NET_TRY(cudaGetLastError());
    // dense 256 -> 12
    NET_TRY(gemm(kOut, L.ld(5), B, split_for(B), MatT{n->g_y, kOut}, MatBias{n->h4, kHidden, kHidden},
                 EpAtomic{n->grads + L.off[5], L.ld(5)}, st, nl));
    NET_TRY(gemm(B, kHidden, kOut, 1, Mat{n->g_y, kOut}, WN{n->wbf + L.offp[5], L.ldp(5)}, EpStore{n->g_h4, kHidden},
                 st, nl));
    k_relu_mask<<<blocks_for((size_t)B * kHidden), 256, 0, st>>>(n->g_h4, n->h4, (size_t)B * kHidden);
    ++*nl;
    NET_TRY(cudaGetLastError());
    // dense 258 -> 256
    NET_TRY(gemm(kHidden, L.ld(4), B, split_for(B), MatT{n->g_h4, kHidden}, MatBias{n->hin, kHin, kHin},
                 EpAtomic{n->grads + L.off[4], L.ld(4)}, st, nl));
    NET_TRY(gemm(B, kHin, kHidden, 1, Mat{n->g_h4, kHidden}, WN{n->wbf + L.offp[4], L.ldp(4)}, EpStore{n->g_hin, kHin},
                 st, nl));
    // global mean
    k_gap_back<<<blocks_for((size_t)B * 64 * kC4), 256, 0, st>>>(n->g_hin, n->g_r[3], B, 64, kC4);
    ++*nl;
    NET_TRY(cudaGetLastError());
    // conv 128 -> 256 on 8 x 8
    NET_TRY(gemm(kC4, L.ld(3), B * 64, split_for(B * 64LL), ReluGradT<kC4>{n->g_r[3], n->r[3]},
                 ConvIn<8, kC3, __nv_bfloat16>{n->pool[2]}, EpAtomic{n->grads + L.off[3], L.ld(3)}, st, nl));
    NET_TRY(gemm(B * 64, kC3, 9 * kC4, 1, DzShift<8, kC4>{n->g_r[3], n->r[3]}, WFlip<kC3, kC4>{n->wbf + L.offp[3], L.ldp(3)},
                 EpStore{n->g_pool[2], kC3}, st, nl));
    k_maxpool_back<<<blocks_for((size_t)B * 64 * kC3), 256, 0, st>>>(n->g_pool[2], n->arg[2], n->g_r[2], B, 16, kC3);
    ++*nl;
    NET_TRY(cudaGetLastError());
    // conv 64 -> 128 on 16 x 16
    NET_TRY(gemm(kC3, L.ld(2), B * 256, split_for(B * 256LL), ReluGradT<kC3>{n->g_r[2], n->r[2]},
                 ConvIn<16, kC2, __nv_bfloat16>{n->pool[1]}, EpAtomic{n->grads + L.off[2], L.ld(2)}, st, nl));
    NET_TRY(gemm(B * 256, kC2, 9 * kC3, 1, DzShift<16, kC3>{n->g_r[2], n->r[2]}, WFlip<kC2, kC3>{n->wbf + L.offp[2], L.ldp(2)},
                 EpStore{n->g_pool[1], kC2}, st, nl));
    k_maxpool_back<<<blocks_for((size_t)B * 256 * kC2), 256, 0, st>>>(n->g_pool[1], n->arg[1], n->g_r[1], B, 32,
                                                                     kC2);
    ++*nl;
    NET_TRY(cudaGetLastError());
    // conv 32 -> 64 on 32 x 32
    NET_TRY(gemm(kC2, L.ld(1), B * 1024, split_for(B * 1024LL), ReluGradT<kC2>{n->g_r[1], n->r[1]},
                 ConvIn<32, kC1, __nv_bfloat16>{n->pool[0]}, EpAtomic{n->grads + L.off[1], L.ld(1)}, st, nl));
    NET_TRY(gemm(B * 1024, kC1, 9 * kC2, 1, DzShift<32, kC2>{n->g_r[1], n->r[1]}, WFlip<kC1, kC2>{n->wbf + L.offp[1], L.ldp(1)},
                 EpStore{n->g_pool[0], kC1}, st, nl));
    k_maxpool_back<<<blocks_for((size_t)B * 1024 * kC1), 256, 0, st>>>(n->g_pool[0], n->arg[0], n->g_r[0], B, 64,
                                                                      kC1);
    ++*nl;
    NET_TRY(cudaGetLastError());
    // conv 8 -> 32 on 64 x 64 (weights only)
    NET_TRY(gemm(kC1, L.ld(0), B * 4096, split_for(B * 4096LL), ReluGradT<kC1>{n->g_r[0], n->r[0]},
                 ConvIn<64, kC0, float>{n->in}, EpAtomic{n->grads + L.off[0], L.ld(0)}, st, nl));
    return APIC_OK;
}

apic_status apic_net_adamw(apic_net* n, float lr, float beta1, float beta2, float eps, float weight_decay, int step,
                           void* stream) {
    if (!n) return net_fail(APIC_EINVAL, "NULL network");
    if (step < 1 || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return net_fail(APIC_EINVAL, "bad optimizer arguments");
    const size_t P = n->L.total;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adamw<<<blocks_for(P), 256, 0, (cudaStream_t)stream>>>(n->params, n->grads, n->m, n->v, n->wbf, P, lr, beta1,
                                                              beta2, eps, weight_decay, c1, c2, n->L);
    ++n->launches;
    NET_TRY(cudaGetLastError());
    return APIC_OK;
}

apic_status apic_net_activation(const apic_net* n, int which, float* h, size_t count) {
    if (!n || !h) return net_fail(APIC_EINVAL, "NULL network or destination");
    const size_t B = (size_t)n->last_batch;
    if (B == 0) return net_fail(APIC_EINVAL, "no forward pass yet");
    if (which < 0 || which > 6) return net_fail(APIC_EINVAL, "which must be in [0, 6]");
    NET_TRY(cudaDeviceSynchronize());
    if (which < 4) {
        const int C[4] = {kC1, kC2, kC3, kC4}, H[4] = {64, 32, 16, 8};
        const size_t sz = B * H[which] * H[which] * C[which];
        if (count != sz) return net_fail(APIC_EINVAL, "activation size mismatch");
        std::vector<uint16_t> tmp(sz);
        NET_TRY(cudaMemcpy(tmp.data(), n->r[which], sz * 2, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < sz; ++i) {
            const uint32_t bits = (uint32_t)tmp[i] << 16;
            std::memcpy(h + i, &bits, 4);
        }
        return APIC_OK;
    }
    const float* src = which == 4 ? n->hin : which == 5 ? n->h4 : n->y;
    const size_t sz = B * (which == 4 ? kHin : which == 5 ? kHidden : kOut);
    if (count != sz) return net_fail(APIC_EINVAL, "activation size mismatch");
    NET_TRY(cudaMemcpy(h, src, sz * 4, cudaMemcpyDeviceToHost));
    return APIC_OK;
}

}  // extern "C"
