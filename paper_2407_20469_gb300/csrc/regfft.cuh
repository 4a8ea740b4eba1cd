// regfft.cuh - register-resident FFTs of length N = 16 B computed by one
// half-warp (16 lanes), for the darkfield correlations.
//
// Cooley-Tukey with N = 16 * B, in two orientations that chain without any
// data exchange between a transform and the next one:
//   alpha: lane t holds x[t + 16 j] (j < B). Step A: DFT_B over j in registers,
//          twiddle W_N^(t k2), padded shared-memory transpose, step B: lane
//          k2 < B runs a DFT_16 over t. Out: lane k2 holds X[k2 + B k1], k1 < 16.
//   beta:  lane u < B holds x[u + B j] (j < 16) - alpha's output layout. Step A:
//          DFT_16 over j, twiddle W_N^(u k2), transpose, step B: lane k2 < 16
//          runs DFT_B over u. Out: lane k2 holds X[k2 + 16 k1] - alpha's input.
// So transform -> pointwise op -> transform of the other orientation needs no
// extra exchange. Small DFTs are unrolled Cooley-Tukey (radix 4, 2, 3) with
// compile-time twiddles; W = exp(-2 pi i / N) forward, conjugate inverse,
// unnormalised. The half-warp's shared area holds max(17 B, 16 (B + 1)) values.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace apic {

// ---- compile-time cos / sin (Taylor series after reduction to [-pi/4, pi/4])
namespace cx {
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
// cos and sin of 2 pi k / N, reduced to an octant by exact symmetries
constexpr void cos_sin_turn(long k, long N, double& c, double& s) {
    long r = ((k % N) + N) % N;          // angle = 2 pi r / N in [0, 2 pi)
    // quadrant q: angle = q pi/2 + a, a in [0, pi/2)
    const long q = (4 * r) / N;
    const long rr = 4 * r - q * N;       // a = (pi / 2) rr / N
    const double a = kPi / 2.0 * (double)rr / (double)N;
    double ca = 0.0, sa = 0.0;
    if (2 * rr <= N) {                   // a <= pi/4
        ca = taylor_cos(a);
        sa = taylor_sin(a);
    } else {                             // use the complement pi/2 - a
        const double b = kPi / 2.0 - a;
        ca = taylor_sin(b);
        sa = taylor_cos(b);
    }
    switch (q) {
        case 0: c = ca; s = sa; break;
        case 1: c = -sa; s = ca; break;
        case 2: c = -ca; s = -sa; break;
        default: c = sa; s = -ca; break;
    }
}
constexpr float wre(long k, long N) { double c = 0, s = 0; cos_sin_turn(k, N, c, s); return (float)c; }
constexpr float wim(long k, long N) { double c = 0, s = 0; cos_sin_turn(k, N, c, s); return (float)(-s); }
}  // namespace cx

template <int I, int End, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < End) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, End>(f);
    }
}

// a * W_N^K (forward W = exp(-2 pi i K / N)); inverse uses conj(W).
template <int N, int K, bool INV>
__device__ __forceinline__ float2 twc(float2 a) {
    constexpr int k = ((K % N) + N) % N;
    if constexpr (k == 0) {
        return a;
    } else if constexpr (4 * k == N) {          // W = -i
        return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    } else if constexpr (2 * k == N) {          // W = -1
        return make_float2(-a.x, -a.y);
    } else if constexpr (4 * k == 3 * N) {      // W = +i
        return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    } else {
        constexpr float c = cx::wre(k, N);
        constexpr float s = INV ? -cx::wim(k, N) : cx::wim(k, N);
        return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

template <int N>
struct Radix {
    static constexpr int R = (N % 4 == 0 && N > 4) ? 4 : ((N % 2 == 0 && N > 2) ? 2 : ((N % 3 == 0 && N > 3) ? 3 : N));
};

// In-place DFT of N values held in registers, natural order in and out.
template <int N, bool INV>
struct DFT {
    static __device__ __forceinline__ void run(float2 (&a)[N]) {
        constexpr int R = Radix<N>::R, M = N / R;
        static_assert(R * M == N && R < N, "unsupported DFT length");
        float2 sub[R][M];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < M; ++q) sub[r][q] = a[r + R * q];
#pragma unroll
        for (int r = 0; r < R; ++r) DFT<M, INV>::run(sub[r]);
        static_for<0, M>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            float2 t[R];
            static_for<0, R>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                t[r] = twc<N, r * k, INV>(sub[r][k]);
            });
            DFT<R, INV>::run(t);
#pragma unroll
            for (int s = 0; s < R; ++s) a[k + M * s] = t[s];
        });
    }
};

template <bool INV>
struct DFT<1, INV> {
    static __device__ __forceinline__ void run(float2 (&)[1]) {}
};

template <bool INV>
struct DFT<2, INV> {
    static __device__ __forceinline__ void run(float2 (&a)[2]) {
        const float2 u = a[0], v = a[1];
        a[0] = cadd(u, v);
        a[1] = csub(u, v);
    }
};

template <bool INV>
struct DFT<3, INV> {
    static __device__ __forceinline__ void run(float2 (&a)[3]) {
        // X1,2 = a0 - (a1 + a2)/2 -/+ i (sqrt(3)/2)(a1 - a2) (forward)
        const float h = 0.86602540378443865f;
        const float2 s = cadd(a[1], a[2]), d = csub(a[1], a[2]);
        const float2 m = make_float2(a[0].x - 0.5f * s.x, a[0].y - 0.5f * s.y);
        const float2 r = INV ? make_float2(-h * d.y, h * d.x) : make_float2(h * d.y, -h * d.x);  // -/+ i h d
        a[0] = cadd(a[0], s);
        a[1] = cadd(m, r);
        a[2] = csub(m, r);
    }
};

template <bool INV>
struct DFT<5, INV> {
    static __device__ __forceinline__ void run(float2 (&a)[5]) {
        // with t1 = a1 + a4, t2 = a2 + a3, t3 = a1 - a4, t4 = a2 - a3 and W = exp(-2 pi i / 5):
        // X1,4 = a0 + c1 t1 + c2 t2 -/+ i (s1 t3 + s2 t4), X2,3 = a0 + c2 t1 + c1 t2 -/+ i (s2 t3 - s1 t4)
        // (forward; c_k = cos(2 pi k / 5), s_k = sin(2 pi k / 5); the inverse swaps the signs of i)
        constexpr float c1 = cx::wre(1, 5), c2 = cx::wre(2, 5), s1 = -cx::wim(1, 5), s2 = -cx::wim(2, 5);
        const float2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]), t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
        const float2 m1 = make_float2(a[0].x + c1 * t1.x + c2 * t2.x, a[0].y + c1 * t1.y + c2 * t2.y);
        const float2 m2 = make_float2(a[0].x + c2 * t1.x + c1 * t2.x, a[0].y + c2 * t1.y + c1 * t2.y);
        const float2 n1 = make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
        const float2 n2 = make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
        // -i n = (n.y, -n.x)
        const float2 r1 = INV ? make_float2(-n1.y, n1.x) : make_float2(n1.y, -n1.x);
        const float2 r2 = INV ? make_float2(-n2.y, n2.x) : make_float2(n2.y, -n2.x);
        a[0] = cadd(a[0], cadd(t1, t2));
        a[1] = cadd(m1, r1);
        a[4] = csub(m1, r1);
        a[2] = cadd(m2, r2);
        a[3] = csub(m2, r2);
    }
};

template <bool INV>
struct DFT<4, INV> {
    static __device__ __forceinline__ void run(float2 (&a)[4]) {
        const float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]), t2 = cadd(a[1], a[3]);
        const float2 d = csub(a[1], a[3]);
        const float2 t3 = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = cadd(t1, t3);
        a[3] = csub(t1, t3);
    }
};

// Half-warp helpers: lane t in [0, 16), the half-warp mask, its shared area hs.
// Twiddles between the steps come from a per-length table in shared memory laid
// out for conflict-free lane access: tw[k2 * 16 + t] = W_N^(t k2) (k2 < B) for
// alpha, followed by tw[16 B + k2 * B + u] = W_N^(u k2) (k2 < 16) for beta;
// W = exp(-2 pi i / N). make_step_twiddles fills it from a plain N-entry table.
struct HalfWarp {
    int t;
    unsigned mask;
    float2* hs;
};

template <int B>
struct HWSize {
    static constexpr int value = (17 * B > 16 * (B + 1) ? 17 * B : 16 * (B + 1));
};
__host__ __device__ constexpr int hw_single_size(int B) { return 17 * B > 16 * (B + 1) ? 17 * B : 16 * (B + 1); }

__device__ __forceinline__ float2 tw_get(const float2* tw, int k, bool inv) {
    const float2 w = tw[k];
    return inv ? make_float2(w.x, -w.y) : w;
}

// Fills the 2 * 16 B step twiddles of length N = 16 B from a plain table W_N^k.
__device__ inline void make_step_twiddles(float2* dst, const float2* plain, int B) {
    const int N = 16 * B;
    for (int i = threadIdx.x; i < 16 * B; i += blockDim.x) {
        const int k2 = i >> 4, t = i & 15;               // alpha: [k2 < B][t < 16]
        dst[i] = plain[(t * k2) % N];
        const int k2b = i / B, u = i - k2b * B;          // beta: [k2 < 16][u < B]
        dst[16 * B + i] = plain[(u * k2b) % N];
    }
}

// alpha: v[j] = x[t + 16 j] -> lanes t < B: o[k1] = X[t + B k1].
template <int B, bool INV>
__device__ __forceinline__ void fft_alpha(float2 (&v)[B], float2 (&o)[16], const HalfWarp& h, const float2* tw) {
    static_assert(B <= 16, "alpha needs B <= 16");
    DFT<B, INV>::run(v);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) h.hs[k2 * 17 + h.t] = cmul(v[k2], tw_get(tw, k2 * 16 + h.t, INV));
    __syncwarp(h.mask);
    // lanes t >= B have no step-B work; they transform a copy of row 0 (discarded)
    const int row = h.t < B ? h.t : 0;
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) o[n1] = h.hs[row * 17 + n1];
    DFT<16, INV>::run(o);
    __syncwarp(h.mask);
}

// beta: lanes u < B: o[j] = x[u + B j] -> all lanes: v[k1] = X[t + 16 k1].
template <int B, bool INV>
__device__ __forceinline__ void fft_beta(float2 (&o)[16], float2 (&v)[B], const HalfWarp& h, const float2* tw) {
    static_assert(B <= 16, "beta needs B <= 16");
    DFT<16, INV>::run(o);           // lanes t >= B transform values they do not store
    if (h.t < B) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) h.hs[k2 * (B + 1) + h.t] = cmul(o[k2], tw_get(tw, 16 * B + k2 * B + h.t, INV));
    }
    __syncwarp(h.mask);
#pragma unroll
    for (int u = 0; u < B; ++u) v[u] = h.hs[h.t * (B + 1) + u];
    DFT<B, INV>::run(v);
    __syncwarp(h.mask);
}

// ---- two transforms of length N = 16 B (2 B <= 16) per half-warp, columns a and b.
// The single-column form leaves lanes t >= B idle in its DFT_16 step; here lanes
// t < B carry column a there and lanes B <= t < 2 B column b. Same step twiddles.
// Half-warp area: alpha 2 B rows of 17; beta two 16 x (B + 1) blocks, the second
// shifted by 8 values so that the two columns' writes fall in different banks.
__host__ __device__ constexpr int hw_pair_size(int B) {
    return 34 * B > 32 * (B + 1) + 8 ? 34 * B : 32 * (B + 1) + 8;
}

// alpha2: va[j] = a[t + 16 j], vb[j] = b[t + 16 j] -> lane t < B: o[k1] = A[t + B k1],
// lane B <= t < 2 B: o[k1] = B[t - B + B k1].
template <int B, bool INV>
__device__ __forceinline__ void fft_alpha2(float2 (&va)[B], float2 (&vb)[B], float2 (&o)[16], const HalfWarp& h,
                                           const float2* tw) {
    static_assert(2 * B <= 16, "alpha2 needs 2 B <= 16");
    DFT<B, INV>::run(va);
    DFT<B, INV>::run(vb);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) {
        const float2 wt = tw_get(tw, k2 * 16 + h.t, INV);
        h.hs[k2 * 17 + h.t] = cmul(va[k2], wt);
        h.hs[(B + k2) * 17 + h.t] = cmul(vb[k2], wt);
    }
    __syncwarp(h.mask);
    const int row = h.t < 2 * B ? h.t : 0;
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) o[n1] = h.hs[row * 17 + n1];
    DFT<16, INV>::run(o);
    __syncwarp(h.mask);
}

// beta2: lane t < 2 B holds o[j] = (t < B ? a : b)[u + B j], u = t mod B -> all
// lanes: va[k1] = A[t + 16 k1], vb[k1] = B[t + 16 k1].
template <int B, bool INV>
__device__ __forceinline__ void fft_beta2(float2 (&o)[16], float2 (&va)[B], float2 (&vb)[B], const HalfWarp& h,
                                          const float2* tw) {
    static_assert(2 * B <= 16, "beta2 needs 2 B <= 16");
    constexpr int kB = 16 * (B + 1) + 8;     // offset of column b's block
    DFT<16, INV>::run(o);
    if (h.t < 2 * B) {
        const int col = h.t >= B, u = h.t - col * B;
        float2* dst = h.hs + col * kB;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) dst[k2 * (B + 1) + u] = cmul(o[k2], tw_get(tw, 16 * B + k2 * B + u, INV));
    }
    __syncwarp(h.mask);
#pragma unroll
    for (int u = 0; u < B; ++u) {
        va[u] = h.hs[h.t * (B + 1) + u];
        vb[u] = h.hs[kB + h.t * (B + 1) + u];
    }
    DFT<B, INV>::run(va);
    DFT<B, INV>::run(vb);
    __syncwarp(h.mask);
}

}  // namespace apic

namespace apic {

// ---- wide transforms: N = 16 B with 16 < B <= 32 (288, 320, 384, 512 points).
// Step A is the same DFT_B in registers; step B has B DFT_16s, so lane t runs two
// of them, rows k2 = t and k2 = t + 16 (slot 0 and slot 1; slot 1 only where t + 16 < B,
// other lanes transform a copy of row t and discard it). Outputs and inputs of the
// second orientation are therefore held in two slots per lane: value o[s][k1] of lane
// t is X[(t + 16 s) + B k1]. Same step twiddles and half-warp area (17 B values) as
// the single form.
template <int B>
struct Slots {
    static constexpr int value = B > 16 ? 2 : 1;
};

// alpha_w: v[j] = x[t + 16 j] (j < B) -> o[s][k1] = X[(t + 16 s) + B k1].
template <int B, bool INV>
__device__ __forceinline__ void fft_alpha_w(float2 (&v)[B], float2 (&o)[2][16], const HalfWarp& h,
                                            const float2* tw) {
    static_assert(B > 16 && B <= 32, "alpha_w needs 16 < B <= 32");
    DFT<B, INV>::run(v);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) h.hs[k2 * 17 + h.t] = cmul(v[k2], tw_get(tw, k2 * 16 + h.t, INV));
    __syncwarp(h.mask);
    const int r1 = h.t + 16 < B ? h.t + 16 : h.t;
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) {
        o[0][n1] = h.hs[h.t * 17 + n1];
        o[1][n1] = h.hs[r1 * 17 + n1];
    }
    DFT<16, INV>::run(o[0]);
    DFT<16, INV>::run(o[1]);
    __syncwarp(h.mask);
}

// beta_w: slot s of lane t (u = t + 16 s < B) holds o[s][j] = x[u + B j] (j < 16) ->
// every lane: v[k1] = X[t + 16 k1] (k1 < B).
template <int B, bool INV>
__device__ __forceinline__ void fft_beta_w(float2 (&o)[2][16], float2 (&v)[B], const HalfWarp& h,
                                           const float2* tw) {
    static_assert(B > 16 && B <= 32, "beta_w needs 16 < B <= 32");
    DFT<16, INV>::run(o[0]);
    DFT<16, INV>::run(o[1]);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int u = h.t + 16 * s;
        if (u < B) {
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) h.hs[k2 * (B + 1) + u] = cmul(o[s][k2], tw_get(tw, 16 * B + k2 * B + u, INV));
        }
    }
    __syncwarp(h.mask);
#pragma unroll
    for (int u = 0; u < B; ++u) v[u] = h.hs[h.t * (B + 1) + u];
    DFT<B, INV>::run(v);
    __syncwarp(h.mask);
}

// One interface for both forms: o[Slots<B>][16], slot s of lane t carrying the row
// t + 16 s of step B (valid where t + 16 s < B).
template <int B, bool INV>
__device__ __forceinline__ void fft_a(float2 (&v)[B], float2 (&o)[Slots<B>::value][16], const HalfWarp& h,
                                      const float2* tw) {
    if constexpr (B > 16)
        fft_alpha_w<B, INV>(v, o, h, tw);
    else
        fft_alpha<B, INV>(v, o[0], h, tw);
}
template <int B, bool INV>
__device__ __forceinline__ void fft_b(float2 (&o)[Slots<B>::value][16], float2 (&v)[B], const HalfWarp& h,
                                      const float2* tw) {
    if constexpr (B > 16)
        fft_beta_w<B, INV>(o, v, h, tw);
    else
        fft_beta<B, INV>(o[0], v, h, tw);
}

}  // namespace apic
