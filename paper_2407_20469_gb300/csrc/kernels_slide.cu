// kernels_slide.cu - whole-slide tiling: windows of the plan's tile size over a
// larger camera image, cutting them into the batch layout and pasting each
// tile's owned part of the reconstructed field back into a slide-sized field.
//
// The paper reconstructs a slide patch by patch (Sec. 2.3, 3.2). No tile here is
// ragged: windows step by `stride` and the last one of each row / column moves
// inward to end at the slide edge, so one plan (one transform size) serves the
// whole slide. Neighbouring windows split their overlap at its middle.
#include <algorithm>
#include <vector>

#include "../../include/apic.h"
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
