// kernels_slide.cu - whole-slide tiling: windows of the plan's tile size over a
// larger camera image, cutting them into the batch layout, and joining the
// reconstructed fields into one slide-sized field, either by pasting each
// tile's owned part or by blending the overlaps.
//
// The paper reconstructs a slide patch by patch (Sec. 2.3, 3.2). No tile here is
// ragged: windows step by `stride` and the last one of each row / column moves
// inward to end at the slide edge, so one plan (one transform size) serves the
// whole slide. Pasting splits each overlap at its middle; blending (Sec. 2.5
// smooths the seams of overlapping fields of view without a rule) first brings
// the tiles to one global phase - each tile keeps the arbitrary constant phase
// of Eq. 5 - from the sums of f_t conj(f_s) over the overlaps with the left and
// upper neighbours, chained along the window grid, then averages with linear
// ramps across each overlap.
#include <algorithm>
#include <vector>

#include "../../include/apic.h"
#include "common.cuh"
#include "internal.cuh"

namespace apic {

// Window starts along one axis of length L (>= tile): 0, stride, 2 stride, ...
// while the window fits, then L - tile; and the owned interval of each window.
static void axis_windows(int L, int tile, int stride, std::vector<int>& start, std::vector<int>& own0,
                         std::vector<int>& own1) {
    start.clear();
    for (int p = 0;; p += stride) {
        if (p + tile >= L) {
            start.push_back(L - tile);
            break;
        }
        start.push_back(p);
    }
    // a start equal to the previous one (L - tile reached exactly) is dropped
    std::vector<int> s;
    for (int v : start)
        if (s.empty() || v > s.back()) s.push_back(v);
    start = s;
    const size_t k = start.size();
    own0.assign(k, 0);
    own1.assign(k, L);
    for (size_t i = 0; i + 1 < k; ++i) {
        const int a = start[i], b = start[i + 1];          // overlap [b, a + tile)
        const int cut = (b + a + tile) / 2;
        own1[i] = cut;
        own0[i + 1] = cut;
    }
}

// d_slide [n_img][Hs][Ws] -> d_tiles [tiles][n_img][h][w]; a window that leaves
// the slide yields a NaN stack (flagged APIC_TILE_BADINPUT downstream).
__global__ void k_cut_tiles(int n_tiles, int n_img, int h, int w, const float* __restrict__ slide, int Hs, int Ws,
                            const int32_t* __restrict__ win, float* __restrict__ out) {
    const size_t per_tile = (size_t)n_img * h * w;
    const size_t total = (size_t)n_tiles * per_tile;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int t = (int)(i / per_tile);
        size_t r = i - (size_t)t * per_tile;
        const int img = (int)(r / ((size_t)h * w));
        r -= (size_t)img * h * w;
        const int y = (int)(r / w), x = (int)(r - (size_t)y * w);
        const int y0 = win[6 * t], x0 = win[6 * t + 1];
        const bool ok = y0 >= 0 && x0 >= 0 && y0 + h <= Hs && x0 + w <= Ws;
        out[i] = ok ? slide[((size_t)img * Hs + y0 + y) * Ws + x0 + x] : __int_as_float(0x7fc00000);
    }
}

// owned part of each tile's field [tiles][u h][u w] -> slide field [u Hs][u Ws]
__global__ void k_paste_fields(int n_tiles, int h, int w, int u, const float2* __restrict__ field,
                               const int32_t* __restrict__ win, int Hs, int Ws, float2* __restrict__ slide) {
    const int H = u * h, W = u * w;
    const size_t per_tile = (size_t)H * W;
    const size_t total = (size_t)n_tiles * per_tile;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int t = (int)(i / per_tile);
        const size_t r = i - (size_t)t * per_tile;
        const int Y = (int)(r / W), X = (int)(r - (size_t)Y * W);
        const int32_t* wv = win + 6 * t;
        const int sy = u * wv[0] + Y, sx = u * wv[1] + X;           // slide output coordinates
        if (sy < u * wv[2] || sy >= u * wv[4] || sx < u * wv[3] || sx >= u * wv[5]) continue;
        if (sy < 0 || sx < 0 || sy >= u * Hs || sx >= u * Ws) continue;
        slide[(size_t)sy * (u * Ws) + sx] = field[i];
    }
}

static int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

// ---- overlap blending of the windows' fields
// Windows are row-major on an n_rows x n_cols grid (apic_slide_windows); window k
// covers [u y0, u y0 + L) x [u x0, u x0 + L) of the output, L = u tile.

// start (low-resolution pixels) of window row i / column j
__device__ __forceinline__ int win_y(const int32_t* win, int cols, int i) { return win[6 * (i * cols)]; }
__device__ __forceinline__ int win_x(const int32_t* win, int j) { return win[6 * j + 1]; }

// sum over the overlap of window k with its left (d = 0) / upper (d = 1) neighbour
// s of f_k conj(f_s): FP32 per thread, FP64 across the block; 0 without neighbour
__global__ void k_blend_corr(int n_tiles, int cols, int u, int L, const float2* __restrict__ field,
                             const int32_t* __restrict__ win, float2* __restrict__ corr) {
    __shared__ double red[64];
    const int k = blockIdx.x >> 1, d = blockIdx.x & 1;
    if (k >= n_tiles) return;
    const int nb = d == 0 ? (k % cols ? k - 1 : -1) : (k >= cols ? k - cols : -1);
    float sr = 0.f, si = 0.f;
    if (nb >= 0) {
        const int ty = u * win[6 * k], tx = u * win[6 * k + 1], sy = u * win[6 * nb], sx = u * win[6 * nb + 1];
        const int ya = max(ty, sy), yb = min(ty + L, sy + L), xa = max(tx, sx), xb = min(tx + L, sx + L);
        const int w = xb - xa;
        const float2* ft = field + (size_t)k * L * L;
        const float2* fs = field + (size_t)nb * L * L;
        if (ya < yb && w > 0)
            for (int idx = threadIdx.x; idx < (yb - ya) * w; idx += blockDim.x) {
                const int Y = ya + idx / w, X = xa + idx % w;
                const float2 a = ft[(size_t)(Y - ty) * L + (X - tx)], b = fs[(size_t)(Y - sy) * L + (X - sx)];
                sr += a.x * b.x + a.y * b.y;                   // a conj(b)
                si += a.y * b.x - a.x * b.y;
            }
    }
    const double tr = block_sum((double)sr, red), ti = block_sum((double)si, red);
    if (threadIdx.x == 0) corr[2 * k + d] = make_float2((float)tr, (float)ti);
}

// exp(-i phi_k): the first row chained left to right, then every column downward.
// 1. every window's step toward its parent, conj(c) / |c| ((1, 0) for c = 0; the left
//    neighbour's correlation in the first row, the upper one's elsewhere), all in parallel
//    (scaled by max(|re|, |im|) first so that tiny correlations do not underflow);
// 2. the first row's prefix product, log-depth in shared memory (FP64) when the row fits
//    the block, else chained by one thread; 3. each column chained downward by its own thread.
__device__ __forceinline__ float2 unit_conj(float2 c) {
    const float m = fmaxf(fabsf(c.x), fabsf(c.y));
    if (!(m > 0.f)) return make_float2(1.f, 0.f);
    const float x = c.x / m, y = c.y / m;
    const float r = 1.f / sqrtf(x * x + y * y);
    return make_float2(x * r, -y * r);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

constexpr int kPhaseThreads = 1024;

__global__ void __launch_bounds__(kPhaseThreads) k_blend_phases(int rows, int cols, const float2* __restrict__ corr,
                                                                 float2* __restrict__ z) {
    __shared__ double2 top[kPhaseThreads];
    const int n = rows * cols, t = threadIdx.x;
    for (int k = t; k < n; k += blockDim.x)
        z[k] = k == 0 ? make_float2(1.f, 0.f) : unit_conj(k < cols ? corr[2 * k] : corr[2 * k + 1]);
    __syncthreads();                                       // z is read across threads below
    const bool scan = cols <= (int)blockDim.x;
    if (scan) {
        if (t < cols) top[t] = make_double2(z[t].x, z[t].y);
        __syncthreads();
        for (int d = 1; d < cols; d <<= 1) {               // inclusive prefix product
            const bool act = t < cols && t >= d;
            double2 v = make_double2(0.0, 0.0);
            if (act) v = cmul(top[t - d], top[t]);
            __syncthreads();
            if (act) top[t] = v;
            __syncthreads();
        }
    } else if (t == 0) {
        double2 v = make_double2(1.0, 0.0);
        for (int j = 1; j < cols; ++j) {
            v = cmul(v, make_double2(z[j].x, z[j].y));
            z[j] = make_float2((float)v.x, (float)v.y);
        }
    }
    __syncthreads();
    for (int j = t; j < cols; j += blockDim.x) {
        double2 v = scan ? top[j] : make_double2(z[j].x, z[j].y);
        z[j] = make_float2((float)v.x, (float)v.y);
        for (int i = 1; i < rows; ++i) {
            const int k = i * cols + j;
            v = cmul(v, make_double2(z[k].x, z[k].y));
            z[k] = make_float2((float)v.x, (float)v.y);
        }
    }
}

// weight of window j (starts s[], n of them, length L) at output position p along one axis
__device__ __forceinline__ float blend_ramp(int sj, int sprev, int snext, bool has_prev, bool has_next, int p, int L) {
    float w = 1.f;
    if (has_prev) {
        const int ov = sprev + L - sj;
        if (ov > 0 && p < sj + ov) w *= ((float)(p - sj) + 0.5f) / (float)ov;
    }
    if (has_next) {
        const int ov = sj + L - snext;
        if (ov > 0 && p >= snext) w *= ((float)(sj + L - p) - 0.5f) / (float)ov;
    }
    return w;
}

// weighted, phase-aligned sum of the windows covering output pixel (Y, X)
__device__ __forceinline__ float2 blend_one(int rows, int cols, int u, int L, const float2* __restrict__ field,
                                            const int32_t* __restrict__ win, const float2* __restrict__ z, int Y,
                                            int X) {
    int lo = 0, hi = rows - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (u * win_y(win, cols, mid) <= Y) lo = mid; else hi = mid - 1;
    }
    const int iy = lo;
    lo = 0;
    hi = cols - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (u * win_x(win, mid) <= X) lo = mid; else hi = mid - 1;
    }
    const int jx = lo;
    float ar = 0.f, ai = 0.f, ws = 0.f;
    for (int i = iy; i >= 0; --i) {
        const int sy = u * win_y(win, cols, i);
        if (sy + L <= Y) break;
        if (sy > Y) continue;
        const float wy = blend_ramp(sy, i > 0 ? u * win_y(win, cols, i - 1) : 0,
                                    i + 1 < rows ? u * win_y(win, cols, i + 1) : 0, i > 0, i + 1 < rows, Y, L);
        for (int j = jx; j >= 0; --j) {
            const int sx = u * win_x(win, j);
            if (sx + L <= X) break;
            if (sx > X) continue;
            const float wx = blend_ramp(sx, j > 0 ? u * win_x(win, j - 1) : 0,
                                        j + 1 < cols ? u * win_x(win, j + 1) : 0, j > 0, j + 1 < cols, X, L);
            const int k = i * cols + j;
            const float2 f = field[(size_t)k * L * L + (size_t)(Y - sy) * L + (X - sx)];
            const float2 zk = z[k];
            const float w = wy * wx;
            ar += w * (f.x * zk.x - f.y * zk.y);
            ai += w * (f.x * zk.y + f.y * zk.x);
            ws += w;
        }
    }
    return ws > 0.f ? make_float2(ar / ws, ai / ws) : make_float2(0.f, 0.f);
}

// output pixel (Y, X) one at a time (odd upsampling or buffers not 16-byte aligned)
__global__ void k_blend(int rows, int cols, int u, int L, const float2* __restrict__ field,
                        const int32_t* __restrict__ win, const float2* __restrict__ z, int Ho, int Wo,
                        float2* __restrict__ out) {
    for (size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i0 < (size_t)Ho * Wo;
         i0 += (size_t)gridDim.x * blockDim.x) {
        const int Y = (int)(i0 / Wo), X = (int)(i0 - (size_t)Y * Wo);
        out[i0] = blend_one(rows, cols, u, L, field, win, z, Y, X);
    }
}

// Output pixel pairs (X, X + 1), X even, over a stripe of kBlendRows rows. With u even,
// window edges in output pixels are even, so both pixels of a pair lie in the same windows
// and their field values are one 16-byte load. The windows covering a pixel along one axis
// are a contiguous run ending at the last one that starts at or before it; each thread
// finds its column run and ramps once, and the block's first kBlendRows threads find the
// row runs and ramps of the stripe into shared memory. A run longer than kMaxCover falls
// back to the per-pixel rule.
constexpr int kMaxCover = 4, kBlendThreads = 128, kBlendRows = 32;

// run of windows (starts u * start(0..count-1), increasing) covering p: last index and length
// (length kMaxCover + 1 when longer than kMaxCover)
template <class Start>
__device__ __forceinline__ int2 cover_run(Start start, int count, int u, int L, int p) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (u * start(mid) <= p) lo = mid; else hi = mid - 1;
    }
    int n = 0;
    while (lo - n >= 0 && n <= kMaxCover) {
        const int s = u * start(lo - n);
        if (s > p || s + L <= p) break;
        ++n;
    }
    return make_int2(lo, n);
}

__global__ void __launch_bounds__(kBlendThreads) k_blend_pairs(int rows, int cols, int u, int L,
                                                                const float2* __restrict__ field,
                                                                const int32_t* __restrict__ win,
                                                                const float2* __restrict__ z, int Ho, int Wo,
                                                                float2* __restrict__ out) {
    __shared__ int s_last[kBlendRows], s_n[kBlendRows], s_sy[kBlendRows][kMaxCover];
    __shared__ float s_wy[kBlendRows][kMaxCover];
    const int Y0 = blockIdx.y * kBlendRows, Y1 = min(Ho, Y0 + kBlendRows);
    auto ystart = [&](int i) { return win_y(win, cols, i); };
    auto xstart = [&](int j) { return win_x(win, j); };
    if (threadIdx.x < kBlendRows && Y0 + (int)threadIdx.x < Y1) {
        const int r = threadIdx.x, Y = Y0 + r;
        const int2 run = cover_run(ystart, rows, u, L, Y);
        s_last[r] = run.x;
        s_n[r] = run.y > kMaxCover ? -1 : run.y;
#pragma unroll
        for (int c = 0; c < kMaxCover; ++c) {
            s_sy[r][c] = 0;
            s_wy[r][c] = 0.f;
            if (c < run.y && run.y <= kMaxCover) {
                const int i = run.x - c, sy = u * ystart(i);
                s_sy[r][c] = sy;
                s_wy[r][c] = blend_ramp(sy, i > 0 ? u * ystart(i - 1) : 0, i + 1 < rows ? u * ystart(i + 1) : 0,
                                        i > 0, i + 1 < rows, Y, L);
            }
        }
    }
    __syncthreads();
    const int X = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (X >= Wo) return;                                   // no synchronisation below
    const int2 cx = cover_run(xstart, cols, u, L, X);
    const int jhi = cx.x, nj = cx.y;
    const bool generic_x = nj > kMaxCover;
    int sxs[kMaxCover];
    float wxa[kMaxCover], wxb[kMaxCover];
#pragma unroll
    for (int c = 0; c < kMaxCover; ++c) {
        sxs[c] = 0;
        wxa[c] = wxb[c] = 0.f;
        if (!generic_x && c < nj) {
            const int j = jhi - c;
            const int sx = u * xstart(j);
            const int sp = j > 0 ? u * xstart(j - 1) : 0, sn = j + 1 < cols ? u * xstart(j + 1) : 0;
            sxs[c] = sx;
            wxa[c] = blend_ramp(sx, sp, sn, j > 0, j + 1 < cols, X, L);
            wxb[c] = blend_ramp(sx, sp, sn, j > 0, j + 1 < cols, X + 1, L);
        }
    }
#pragma unroll 2
    for (int Y = Y0; Y < Y1; ++Y) {
        const int r = Y - Y0, ni = s_n[r];
        float4 o;
        if (generic_x || ni < 0) {
            const float2 a = blend_one(rows, cols, u, L, field, win, z, Y, X);
            const float2 b = blend_one(rows, cols, u, L, field, win, z, Y, X + 1);
            o = make_float4(a.x, a.y, b.x, b.y);
        } else {
            float ar0 = 0.f, ai0 = 0.f, ws0 = 0.f, ar1 = 0.f, ai1 = 0.f, ws1 = 0.f;
#pragma unroll
            for (int ci = 0; ci < kMaxCover; ++ci) {
                if (ci < ni) {
                    const int i = s_last[r] - ci, sy = s_sy[r][ci];
                    const float wy = s_wy[r][ci];
#pragma unroll
                    for (int c = 0; c < kMaxCover; ++c) {
                        if (c < nj) {
                            const int k = i * cols + jhi - c;
                            const float4 f = __ldcs(reinterpret_cast<const float4*>(
                                field + (size_t)k * L * L + (size_t)(Y - sy) * L + (X - sxs[c])));
                            const float2 zk = z[k];
                            const float w0 = wy * wxa[c], w1 = wy * wxb[c];
                            ar0 += w0 * (f.x * zk.x - f.y * zk.y);
                            ai0 += w0 * (f.x * zk.y + f.y * zk.x);
                            ws0 += w0;
                            ar1 += w1 * (f.z * zk.x - f.w * zk.y);
                            ai1 += w1 * (f.z * zk.y + f.w * zk.x);
                            ws1 += w1;
                        }
                    }
                }
            }
            o = make_float4(ws0 > 0.f ? ar0 / ws0 : 0.f, ws0 > 0.f ? ai0 / ws0 : 0.f,
                            ws1 > 0.f ? ar1 / ws1 : 0.f, ws1 > 0.f ? ai1 / ws1 : 0.f);
        }
        __stcs(reinterpret_cast<float4*>(out + (size_t)Y * Wo + X), o);
    }
}

cudaError_t launch_blend(const DevPlan& P, int n_tiles, int rows, int cols, const float2* field, const int32_t* win,
                         int Hs, int Ws, float2* corr, float2* z, float2* out, cudaStream_t st) {
    const int u = P.H / P.h, L = P.H;
    k_blend_corr<<<2 * n_tiles, 256, 0, st>>>(n_tiles, cols, u, L, field, win, corr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_blend_phases<<<1, kPhaseThreads, 0, st>>>(rows, cols, corr, z);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int Ho = u * Hs, Wo = u * Ws;
    const bool pairs = u % 2 == 0 && (((uintptr_t)field | (uintptr_t)out) & 15) == 0;
    if (pairs) {
        const dim3 grid((unsigned)((Wo / 2 + kBlendThreads - 1) / kBlendThreads),
                        (unsigned)((Ho + kBlendRows - 1) / kBlendRows));
        k_blend_pairs<<<grid, kBlendThreads, 0, st>>>(rows, cols, u, L, field, win, z, Ho, Wo, out);
    } else {
        k_blend<<<grid_for((size_t)Ho * Wo), 256, 0, st>>>(rows, cols, u, L, field, win, z, Ho, Wo, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_cut_tiles(const DevPlan& P, int n_tiles, const float* slide, int Hs, int Ws, const int32_t* win,
                             float* out, cudaStream_t st) {
    const size_t total = (size_t)n_tiles * P.n_img * P.h * P.w;
    if (total == 0) return cudaSuccess;
    k_cut_tiles<<<grid_for(total), 256, 0, st>>>(n_tiles, P.n_img, P.h, P.w, slide, Hs, Ws, win, out);
    return cudaGetLastError();
}

cudaError_t launch_paste_fields(const DevPlan& P, int n_tiles, const float2* field, const int32_t* win, int Hs,
                                int Ws, float2* slide, cudaStream_t st) {
    const int u = P.H / P.h;
    const size_t total = (size_t)n_tiles * P.H * P.W;
    if (total == 0) return cudaSuccess;
    k_paste_fields<<<grid_for(total), 256, 0, st>>>(n_tiles, P.h, P.w, u, field, win, Hs, Ws, slide);
    return cudaGetLastError();
}

}  // namespace apic

extern "C" apic_status apic_slide_windows(int slide_h, int slide_w, int tile, int stride, int32_t* h_windows,
                                          int capacity, int* n_windows) {
    if (!n_windows) return (apic_status)apic::record_error(APIC_EINVAL, "NULL n_windows");
    *n_windows = 0;
    if (tile < 1 || slide_h < tile || slide_w < tile)
        return (apic_status)apic::record_error(APIC_EINVAL, "the slide must be at least one tile in each direction");
    if (stride < 1 || stride > tile)
        return (apic_status)apic::record_error(APIC_EINVAL, "stride must be in [1, tile]");
    std::vector<int> ys, oy0, oy1, xs, ox0, ox1;
    apic::axis_windows(slide_h, tile, stride, ys, oy0, oy1);
    apic::axis_windows(slide_w, tile, stride, xs, ox0, ox1);
    const long long count = (long long)ys.size() * (long long)xs.size();
    if (count > 0x7fffffff) return (apic_status)apic::record_error(APIC_EINVAL, "too many windows");
    *n_windows = (int)count;
    if (!h_windows) return APIC_OK;
    if (capacity < count) return (apic_status)apic::record_error(APIC_EINVAL, "capacity smaller than the window count");
    size_t k = 0;
    for (size_t i = 0; i < ys.size(); ++i)
        for (size_t j = 0; j < xs.size(); ++j, ++k) {
            int32_t* w = h_windows + 6 * k;
            w[0] = ys[i];
            w[1] = xs[j];
            w[2] = oy0[i];
            w[3] = ox0[j];
            w[4] = oy1[i];
            w[5] = ox1[j];
        }
    return APIC_OK;
}
