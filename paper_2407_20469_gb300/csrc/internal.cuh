// internal.cuh - device-side view of a plan and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct apic_net;

namespace apic {

constexpr int kThreads = 512;        // threads per block of the transform kernels
constexpr int kChunk = 4096;         // complex elements per shared-memory chunk buffer
// Work counters of a plan (unsigned long long): [1] CG iterations, [2] darkfield solves,
// [4 + i] CG iterations of used darkfield image i (processing order), i < kCountedImages.
constexpr int kCountedImages = 256;
constexpr int kCounters = 4 + kCountedImages;

// One darkfield image admitted by the geometry, in processing order.
struct DevDF {
    int led, kx, ky;
    int N, M, NP;                    // |U|, |Q|, |P|
    int u_off, q_off, p_off;         // offsets into the concatenated point arrays
    int uy0, uy1, qy0, qy1, py0, py1;  // band of rows (signed y) of each set
    int urp, qrp, prp;               // offsets into the concatenated row-pointer array
    int qmask_off;                   // offset of the Q-membership bit rows (register grid)
    int tr;                          // 1: solved transposed (point sets and image with x <-> y)
    int by;                          // column grid of the solve: 16 by points (register kernel)
    int bx;                          // row grid of the solve: 16 bx points (register kernel)
};

struct DevPlan {
    int h, w, H, W, n_bf, n_df, n_img;
    int npup, nap, nrows, m, n_used;
    int mr;                          // register-FFT correlation grid (16 B), 0 if unsupported; 512: the
                                     // wide kernel of 512-pixel tiles (P * P on the camera grid)
    int qmask_words;                 // Q membership words per band row (8; 16 for the wide kernel)
    int max_mx, max_mxy;             // wide kernel: largest row grid and row x column grid of the used images
    int band_u, band_p, band_q;      // largest U, P and Q row bands of the used images
    int max_N, max_M;
    float Rx, Ry;
    int pup_ax, pup_ay;
    // pupil
    const int* pup_x;
    const int* pup_y;
    const int* pup_lut;              // (2 pup_ay + 1)(2 pup_ax + 1)
    const int* pup_rowptr;           // rows -pup_ay..pup_ay of the pupil list
    const int* led_x;
    const int* led_y;
    const int* led_pup;              // NA-matching LED -> pupil index
    // aberration rows
    const int* row_il;               // i | (l << 16)
    const int* row_pi;
    const int* row_pl;
    const int* row_nx;
    const int* row_ny;
    const float* row_A;              // [rows][12]
    const double* Lval;              // 12 x 12 lower Cholesky factors
    const double* Lgrad;
    // aperture
    const int* ap_x;
    const int* ap_y;
    const uint8_t* ap_bf;
    const int* st_ptr;
    const int* st_img;
    const int* st_pup;
    int ap_y0, ap_y1;
    const int* ap_rowptr;            // rows ap_y0..ap_y1
    int ap_x0, ap_x1;
    const int* ap_colptr;            // columns ap_x0..ap_x1 of the aperture list sorted by (x, y)
    const int* ap_cole;              // aperture point of each entry of that order
    // darkfield
    const DevDF* df;
    const int* dU_x; const int* dU_y; const int* dU_pup; const int* dU_ap;
    const int* dP_x; const int* dP_y; const int* dP_pup; const int* dP_ap;
    const int* dQ_x; const int* dQ_y;
    const int* d_rowptr;
    const unsigned* d_qmask;         // per used image: Q band rows x 8 words of two 16-bit lane masks
                                     // (lane t, bit k1: x index t + (mr / 16) k1 is in Q; the wide
                                     // kernel: 16 words, lane-slot t + 16 s)
    // twiddles
    const float2* tw_n;              // n = h = w
    const float2* tw_m;
    const float2* tw_N;              // N = H = W
    const float2* tw_r;              // mr
    const float2* tw_y6;             // 96, 128, 144, 160: shorter grids of the register darkfield
    const float2* tw_y8;
    const float2* tw_y9;
    const float2* tw_y10;
    const float2* tw_w12;            // 192, 256, 288, 320: row and column grids of the wide kernel
    const float2* tw_w16;
    const float2* tw_w18;
    const float2* tw_w20;
};

// Scratch sizes and grids decided at plan creation.
struct Launch {
    int grid_kk, grid_ab, grid_df, grid_syn, grid_sim;
    size_t smem_kk, smem_df, smem_syn, smem_sim;
    int grid_synr;                   // register-transform synthesis (output sides 512, 1024), 0: not used
    size_t smem_synr;
};

// Kernel launchers (return cudaError_t of the launch).
// learned != 0: low-contrast tiles get APIC_TILE_LEARNED instead of APIC_TILE_BACKGROUND.
cudaError_t launch_background(const DevPlan& P, int n_tiles, const float* I, float* c2, int32_t* status,
                              float bg_thresh2, cudaStream_t st, int learned = 0);
cudaError_t launch_kk(const DevPlan& P, const Launch& L, int n_tiles, const float* I, float2* xdisc,
                      float2* scratch, const int32_t* status, cudaStream_t st);
// Kramers-Kronig kernels on an explicit grid (each block uses h * w scratch values):
// shared-memory Stockham version, and the register-FFT version (n = 16 BN, BN in 4, 8, 16).
cudaError_t launch_kk_grid(const DevPlan& P, int grid, size_t smem, int n_tiles, const float* I, float2* xdisc,
                           float2* scratch, const int32_t* status, cudaStream_t st);
size_t kkr_smem_bytes(int BN);
int configure_kkr(int BN, size_t smem);
cudaError_t launch_kk_reg(const DevPlan& P, int grid, size_t smem, int n_tiles, const float* I, float2* xdisc,
                          float2* scratch, const int32_t* status, cudaStream_t st);
// Measured FMA throughput (flop/s) of the current device's CUDA cores, FP32 or FP64 (kernels_peak.cu).
cudaError_t measure_fma_rate(int precision, double* flops_per_s);
// Static scratch of the allocation-free entry point (kernels_noalloc.cu).
size_t noalloc_scratch_bytes();
cudaError_t noalloc_scratch(int device, float2** out);
// c0 [tiles][15] learned coefficients or NULL; warm: also refine from c0 and keep the lower residual.
cudaError_t launch_aberration(const DevPlan& P, const Launch& L, int n_tiles, const float2* xdisc, float* zern,
                              float* beta_scratch, int passes, int32_t* status, cudaStream_t st,
                              const float* c0 = nullptr, int warm = 0);
cudaError_t launch_phase(const DevPlan& P, int n_tiles, const float* zern, float* phi, cudaStream_t st);
cudaError_t launch_stitch(const DevPlan& P, int n_tiles, const float2* xdisc, const float* phi, float2* spec,
                          const int32_t* status, cudaStream_t st);
cudaError_t launch_darkfield(const DevPlan& P, const Launch& L, int n_tiles, const float* I, const float* phi,
                             float2* spec, void* scratch, size_t scratch_per_block, int iters, float tol,
                             int32_t* status, unsigned long long* counters, cudaStream_t st);
cudaError_t launch_synthesize(const DevPlan& P, const Launch& L, int n_tiles, const float2* spec, float2* field,
                              const int32_t* status, cudaStream_t st);
// Register-transform synthesis for output side H = 32 B (B in 16, 32): dynamic shared memory
// and blocks per SM (0: unsupported side or failure).
size_t synr_smem_bytes(int H);
int configure_synr(int H, size_t smem);
cudaError_t launch_pupil(const DevPlan& P, int n_tiles, const float* phi, float2* pupil, const int32_t* status,
                         cudaStream_t st);
cudaError_t launch_sim(const DevPlan& P, const Launch& L, int n_tiles, const float2* obj, const float* phi,
                       float photons, unsigned long long seed, float* I, float2* ohat_scratch, cudaStream_t st);

size_t df_scratch_bytes(const DevPlan& P);

// register-FFT darkfield kernel (m = 16 B, n = 16 BN)
size_t dfr_smem_bytes(int B, int BN, int band_u, int band_q, int max_N);
size_t dfr_scratch_bytes(const DevPlan& P);
int configure_dfr(int B, int BN, size_t smem);
// work: a device int the launcher zeroes on `st`; blocks take tiles from it one at a time
// (NULL: tiles by stride)
cudaError_t launch_darkfield_reg(const DevPlan& P, int grid, size_t smem, int n_tiles, const float* I,
                                 const float* phi, float2* spec, void* scratch, size_t per_block, int iters,
                                 float tol, int32_t* status, unsigned long long* counters, int* work,
                                 cudaStream_t st);

// wide darkfield kernel of 512-pixel tiles (kernels_dfw.cu)
size_t dfw_smem_bytes(int max_N, int band);   // band: max of the U, P and Q row bands
size_t dfw_scratch_bytes(const DevPlan& P);
// tile slots (clusters of K blocks, K in 1, 2, 4) that run at once; grid = tile slots
int configure_dfw(size_t smem, int K);
cudaError_t launch_darkfield_wide(const DevPlan& P, int K, int grid, size_t smem, int n_tiles, const float* I,
                                  const float* phi, float2* spec, void* scratch, size_t per_block, int iters,
                                  float tol, int32_t* status, unsigned long long* counters, int* work,
                                  cudaStream_t st);

// Network features (net.cu): feat [n_tiles][64][64][8] from the first 8 images
// of each stack; `scratch` holds h * 64 complex values per block of `grid`.
cudaError_t launch_features(const DevPlan& P, int grid, int n_tiles, const float* I, float* feat, float2* scratch,
                            cudaStream_t st);
size_t feature_floats();
// Network forward on B tiles (net.cu); out15 [B][15].
cudaError_t net_predict(struct ::apic_net* n, int B, const float* feat, const float* uv, float* out15,
                        cudaStream_t st);
int net_max_batch(const struct ::apic_net* n);
long long net_launches(const struct ::apic_net* n);
// Whole-slide tiling (kernels_slide.cu): windows [tiles][6] = y0, x0, oy0, ox0, oy1, ox1.
cudaError_t launch_cut_tiles(const DevPlan& P, int n_tiles, const float* slide, int Hs, int Ws, const int32_t* win,
                             float* out, cudaStream_t st);
cudaError_t launch_paste_fields(const DevPlan& P, int n_tiles, const float2* field, const int32_t* win, int Hs,
                                int Ws, float2* slide, cudaStream_t st);
cudaError_t launch_blend(const DevPlan& P, int n_tiles, int rows, int cols, const float2* field, const int32_t* win,
                         int Hs, int Ws, float2* corr, float2* z, float2* out, cudaStream_t st);
// Records the message returned by apic_last_error (apic.cu).
int record_error(int status, const char* msg);

// Sets the dynamic shared-memory limit of a transform kernel and returns its
// resident blocks per SM (0 on error). which: 0 kk, 1 aberration, 2 darkfield,
// 3 synthesis, 4 simulated images, 5 object transform.
int configure_kernel(int which, size_t smem);

}  // namespace apic
