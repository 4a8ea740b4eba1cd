/*
 * apic.h - C interface of the GB300 per-tile APIC reconstruction library.
 *
 * APIC (angular ptychographic imaging with a closed-form solution), as used by
 * WSI-APIC (arXiv 2407.20469, Sec. 2.3): from a stack of low-resolution
 * intensity images of one slide tile - NA-matching images first, darkfield
 * images after - recover the complex high-resolution field and the pupil
 * aberration. Every tile of a batch is independent; all per-tile arithmetic
 * runs in this library's CUDA kernels (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named d_* are DEVICE pointers (the current CUDA device at the
 *   call); h_* are HOST pointers. The caller owns every buffer it passes; the
 *   library owns only the plan and the plan's workspace.
 * - Complex arrays are interleaved float pairs (re, im), i.e. complex64.
 * - Calls that take a stream are asynchronous and stream-ordered: they enqueue
 *   work on `stream` (a cudaStream_t passed as void*, NULL = legacy default
 *   stream) and return once it is enqueued. Device-side results are valid
 *   after the stream reaches that point.
 * - A host return code other than APIC_OK means nothing was enqueued (argument
 *   or set-up error) or a launch failed (APIC_ECUDA). Numerical trouble in a
 *   tile never traps: it is reported per tile in d_tile_status.
 * - A plan may be used from one host thread at a time; concurrent calls on the
 *   same plan from several streams race on its workspace.
 *
 * Frequencies and layouts
 * -----------------------
 * A plan serves one tile-size class h x w (low-resolution pixels of pitch
 * pixel_um in the sample plane) and upsampling u: the output grid is
 * (u h) x (u w) with pitch pixel_um / u. The frequency step is 1/(w dx) along
 * x and 1/(h dx) along y on both grids. Spectra are Fourier-series
 * coefficients (DFT / number of samples); signed integer frequency k of an
 * n-point axis lives at index k mod n. Illumination wave-vectors are snapped
 * to the integer grid at plan creation (apic_plan_query reports the result).
 */
#ifndef APIC_H
#define APIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes of every entry point. */
typedef enum {
    APIC_OK = 0,
    APIC_EINVAL = 1,      /* bad argument (NULL, size, count, layout)            */
    APIC_ENOMEM = 2,      /* device or host allocation failed                    */
    APIC_ECUDA = 3,       /* a CUDA call or kernel launch failed                 */
    APIC_EGEOMETRY = 4,   /* illumination geometry unusable for this tile size  */
    APIC_EINTERNAL = 5,   /* library bug (an invariant did not hold)             */
    APIC_ENOTCONV = 6     /* all outputs written, but a darkfield solve of some
                             tile stopped above its tolerance (its status word
                             has APIC_TILE_NOTCONV); returned by the synchronous
                             host call apic_reconstruct_host only              */
} apic_status;

/* Per-tile status words written to d_tile_status (bit flags, 0 = clean). */
#define APIC_TILE_OK          0
#define APIC_TILE_BACKGROUND  1   /* below the background-contrast threshold (Sec. 3.2) */
#define APIC_TILE_NOTCONV     2   /* a darkfield solve stopped above its tolerance      */
#define APIC_TILE_BADINPUT    4   /* non-finite or negative intensity in the stack      */
#define APIC_TILE_LEARNED     8   /* low contrast: pupil taken from the network, tile
                                     reconstructed with it (apic_reconstruct_learned)   */
#define APIC_TILE_WARM       16   /* the solve started from the network's coefficients
                                     left the smaller residual and was kept             */

/* Plan flags. */
#define APIC_SKIP_BACKGROUND  1   /* background tiles: outputs zeroed, no reconstruction */
#define APIC_HOST_ONLY        2   /* build the geometry only: no device memory, no CUDA
                                     calls; only apic_plan_query / apic_plan_table /
                                     apic_plan_df_set / apic_plan_destroy accept it */
#define APIC_LEGACY_KERNELS   4   /* Kramers-Kronig and darkfield stages with the shared-
                                     memory Stockham kernels (darkfield on a power-of-two
                                     grid) instead of the register-FFT kernels (for
                                     comparison)                                          */

/* Number of Zernike coefficients per tile (Noll j = 1..15; j = 1..3 always 0). */
#define APIC_N_ZERNIKE 15

typedef struct {
    int tile_h, tile_w;          /* low-resolution tile size of this plan (>= 16, powers of 2) */
    int n_bf, n_df;              /* NA-matching then darkfield image counts                  */
    const float* h_kx;           /* host [n_bf + n_df] transverse illumination k, cycles/um */
    const float* h_ky;
    float na;                    /* objective numerical aperture (0.25)                      */
    float wavelength_um;         /* 0.52                                                      */
    float pixel_um;              /* camera pixel in the sample plane (0.345)                  */
    int upsample;                /* output upsampling factor u (2; 3 for the paper's set-up
                                    size): u tile_h must be 2^k or 3 * 2^k, at most 3072      */
    int max_tiles;               /* largest n_tiles of one call; larger calls are chunked     */
    int df_iters;                /* CGLS iterations per darkfield image (<= 0: 40)            */
    float df_tol;                /* CG stop: ||C^H r|| <= df_tol ||C^H b|| (<= 0: 3e-4, which
                                    keeps the darkfield-only spectrum within ~6e-4 relative
                                    L2 of the exact least-squares solution)                  */
    int ab_passes;               /* value passes of the aberration solve (< 0: 2)             */
    float bg_contrast;           /* background threshold on RMS contrast (Sec. 3.2; 0.02)     */
    int flags;                   /* APIC_SKIP_BACKGROUND                                       */
} apic_params;

typedef struct apic_plan apic_plan;
typedef struct apic_net apic_net;

/* Sizes of a plan's fixed index sets (for callers laying out stage buffers). */
typedef struct {
    int tile_h, tile_w, out_h, out_w;
    int n_bf, n_df;
    int n_pupil;           /* grid points inside the pupil (Circ_NA of Eq. 1)              */
    int n_aperture;        /* object frequencies of the final synthetic aperture           */
    int n_rows;            /* rows of the aberration system D phi = beta (Eq. 10)          */
    int n_df_used;         /* darkfield images the geometry admits (Sec. 4: <= 42% unknown) */
    int fft_m;             /* grid of the darkfield correlations                            */
    double pupil_rx, pupil_ry;   /* pupil radius in grid steps along x and y              */
    int df_wave;           /* tiles whose darkfield solves run at once (one per block or
                              cluster); 0 for a host-only plan                          */
} apic_plan_info;

/* Human-readable name of a return code. Never NULL. */
const char* apic_status_string(apic_status s);

/* Message describing the last error returned on the calling host thread. Never NULL. */
const char* apic_last_error(void);

/*
 * Measured FMA throughput of the current device's CUDA cores, in flop/s (one
 * FMA = 2 flops), for precision 32 (FP32) or 64 (FP64): a kernel of
 * independent multiply-add chains on every SM, the best of three timed
 * launches after one warm-up (CUDA events on the legacy default stream, which
 * it synchronises). The denominator of the rooflines of the library's
 * ALU-bound kernels; the paper has no counterpart. Changes no device setting.
 * Errors: APIC_EINVAL (other precision, NULL output), APIC_ECUDA.
 */
apic_status apic_measure_fma_rate(int precision, double* h_flops_per_s);

/*
 * Build a plan: snap the illumination to the grid (NA-matching LEDs keep the
 * DC term on the edge of the shifted pupil, Sec. 2.3), enumerate the overlap
 * sets S_il (Eq. 8), the darkfield sets U, P, Q (Eq. 11-13, images taken by
 * increasing |k|), upload the index tables and allocate workspace for
 * max_tiles tiles on the current device. *out receives the plan.
 * Errors: APIC_EINVAL (NULL or out-of-range field), APIC_EGEOMETRY (an
 * NA-matching LED has no admissible grid point, or the spectrum leaves the
 * output grid), APIC_ENOMEM, APIC_ECUDA.
 */
apic_status apic_plan_create(const apic_params* params, apic_plan** out);

/* Free a plan and its device memory (synchronises the device first). NULL is a no-op. */
apic_status apic_plan_destroy(apic_plan* plan);

/* Sizes of the plan's index sets. */
apic_status apic_plan_query(const apic_plan* plan, apic_plan_info* info);

/*
 * Copy one of the plan's integer tables to host memory (int32):
 *   APIC_TABLE_LEDS      [n_bf + n_df][2] snapped (kx, ky) of each LED
 *   APIC_TABLE_PUPIL     [n_pupil][2]     camera frequencies k inside the pupil
 *   APIC_TABLE_APERTURE  [n_aperture][2]  object frequencies of the aperture
 * `count` is the number of int32 the destination holds; APIC_EINVAL if short.
 */
#define APIC_TABLE_LEDS      0
#define APIC_TABLE_PUPIL     1
#define APIC_TABLE_APERTURE  2
apic_status apic_plan_table(const apic_plan* plan, int which, int32_t* h_dst, size_t count);

/*
 * Index sets of darkfield image `index` in processing order (Eq. 11-13), all
 * images including skipped ones, as int32 pairs in the pupil frame c = K + k_j:
 *   which 0: U (unknown), 1: P (known), 2: Q (lags), each sorted by (y, x).
 * h_meta (may be NULL) receives {led index, used (0/1), |U|, |P|, |Q|}.
 * h_dst may be NULL to query the sizes only; otherwise it holds `count` int32.
 */
apic_status apic_plan_df_set(const apic_plan* plan, int index, int which, int32_t* h_dst, size_t count,
                             int32_t* h_meta);

/*
 * Frame and transform grid of the darkfield solve of image `index` (processing
 * order; an implementation choice that leaves Eq. 13 unchanged): h_grid[3]
 * receives {1 if the image is solved with x and y swapped else 0, row grid
 * points, column grid points of the register-FFT kernel in the solve frame,
 * both exact for the correlations of that image (0 when the plan has no
 * register grid)}; {0, 0, 0} for a skipped image. Accepts a host-only plan.
 */
apic_status apic_plan_df_grid(const apic_plan* plan, int index, int32_t* h_grid);

/*
 * Sets the register-kernel grid of darkfield image `index` to mx row points x
 * my column points, one of the supported pairs 192 x {96, 128, 144, 192},
 * 160 x {96, 128} and 144 x 144 (plans whose register grid is 192 points), and
 * rebuilds the plan's device tables (synchronises the device). APIC_EINVAL if
 * the image is skipped, the pair is unsupported or it would alias the image's
 * correlations. The plan's own choice is the cheapest exact pair; this lets a
 * caller (or a test) run any other. The device tables move, so work with this
 * plan captured in a CUDA graph before the call must be captured again; no
 * call with the plan may be in flight on another host thread.
 */
apic_status apic_plan_set_df_grid(apic_plan* plan, int index, int mx, int my);

/*
 * Whole per-tile reconstruction (Sec. 2.3, Fig. 2), for n_tiles tiles:
 *   d_intensity  [n_tiles][n_bf + n_df][h][w] float32 intensity stacks
 *   d_field      [n_tiles][u h][u w] complex64 out: high-resolution field
 *   d_zernike    [n_tiles][15] float32 out: Noll coefficients (rad) of phi
 *   d_pupil      [n_tiles][h][w] complex64 out, or NULL: Circ(k) exp(j phi(k)),
 *                frequency k at index k mod n
 *   d_tile_status [n_tiles] int32 out, or NULL: APIC_TILE_* bits
 * Steps: background test (Sec. 3.2), Kramers-Kronig recovery (Eq. 4-7),
 * aberration solve (Eq. 8-10), correction and stitching, darkfield extension
 * (Eq. 11-13), inverse transform. The global phase of the field is the
 * phase gauge of Eq. 5 (mean phase of the recovered fields set to zero).
 * Batches above max_tiles are processed in chunks. When a chunk is not a
 * whole number of darkfield waves (one tile per block) and its last partial
 * wave holds at most half a wave, that wave's darkfield solves run first, on
 * a second stream the plan owns, forked from and joined back to `stream`
 * (stream capture follows the fork), while the other tiles' earlier stages
 * run on the remaining SMs; a larger partial wave simply ends the darkfield
 * stage. Results are identical in every order.
 */
apic_status apic_reconstruct_batch(apic_plan* plan, int n_tiles, const float* d_intensity,
                                   float* d_field, float* d_zernike, float* d_pupil,
                                   int32_t* d_tile_status, void* stream);

/*
 * Work counters of a plan since creation or the last reset, for throughput
 * accounting: h_out[0] kernel launches issued, h_out[1] CGLS iterations run,
 * h_out[2] darkfield least-squares solves run, h_out[3 + i] the CGLS
 * iterations of the i-th used darkfield image (in the processing order of
 * apic_plan_df_set / apic_plan_df_grid, skipped images not counted; the first
 * 256 used images).
 * Up to n values are written.
 * Synchronises the device (reads a device counter); reset != 0 zeroes them.
 */
apic_status apic_plan_counters(apic_plan* plan, int64_t* h_out, int n, int reset);

/*
 * Per-stage timing of apic_reconstruct_batch with CUDA events recorded on the
 * call's stream around every stage launch (a ring of 1024 calls; calls made
 * while the stream is being captured into a graph are not timed).
 * apic_plan_timing(plan, 1) creates the events, (plan, 0) stops recording.
 * apic_plan_stage_ms synchronises the device and writes, for stage s, the
 * summed milliseconds over the recorded calls to h_ms[s] (s: 0 background,
 * 1 Kramers-Kronig, 2 aberration, 3 stitch, 4 darkfield, 5 synthesis,
 * 6 pupil; n <= 7 values) and the number of calls to *h_calls (may be NULL);
 * reset != 0 clears the ring.
 */
apic_status apic_plan_timing(apic_plan* plan, int enable);
apic_status apic_plan_stage_ms(apic_plan* plan, double* h_ms, int n, int32_t* h_calls, int reset);

/*
 * apic_reconstruct_batch from and to HOST memory, pipelined. A batch of up to
 * max_tiles tiles that has a partial GPU-wide darkfield wave (or fits four
 * waves) is one chunk with its copies woven into the reconstruction's own
 * order: the partial wave's intensities first, the others in up to 16 parts
 * whose earlier stages start as each part lands, and every darkfield round's
 * fields copied out as soon as they are synthesized (the first 32 rounds; the
 * rest when the computation ends). Other batches go in chunks (the first one
 * wave, the rest up to four waves or max_tiles): while one chunk is
 * reconstructed the next chunk's intensities are copied in and the previous
 * chunk's results copied out. Three internal streams; device staging buffers
 * allocated on first use and kept: one set for max_tiles tiles (inputs,
 * fields, coefficients, status) when that leaves a quarter of the free device
 * memory (at least 1 GiB), else for one chunk (then every batch is chunked),
 * and a second set of one chunk once a batch is chunked. For the copies to overlap the host buffers must be
 * pinned (cudaHostAlloc / cudaHostRegister); pageable buffers work but
 * serialise. Returns when all results are in host memory.
 *   h_intensity [n_tiles][n_bf + n_df][h][w] f32, h_field [n_tiles][u h][u w]
 *   complex64, h_zernike [n_tiles][15] f32, h_tile_status [n_tiles] or NULL.
 * Returns APIC_ENOTCONV (outputs complete) when h_tile_status is given and some
 * tile's word has APIC_TILE_NOTCONV: its field is the darkfield solve's last
 * iterate, usable but above the CG tolerance.
 */
apic_status apic_reconstruct_host(apic_plan* plan, int n_tiles, const float* h_intensity, float* h_field,
                                  float* h_zernike, int32_t* h_tile_status);

/* ---- Stages of apic_reconstruct_batch, for testing and custom pipelines ---- */

/*
 * Background statistic (Sec. 3.2): per tile, the mean over the NA-matching
 * images of var(I)/mean(I)^2 (squared RMS contrast), written to d_contrast2
 * [n_tiles] float32, and d_tile_status [n_tiles] set to APIC_TILE_BACKGROUND
 * where it is below bg_contrast^2 (else 0), with APIC_TILE_BADINPUT where
 * the stack holds a negative or non-finite value.
 */
apic_status apic_background(apic_plan* plan, int n_tiles, const float* d_intensity,
                            float* d_contrast2, int32_t* d_tile_status, void* stream);

/*
 * Kramers-Kronig recovery (Eq. 4-7) of every NA-matching image:
 *   d_xdisc [n_tiles][n_bf][n_pupil] complex64 out: X_i(K) = S'_i(K) exp(-j theta_i)
 *   at K = k_p - k_i for the pupil points k_p (APIC_TABLE_PUPIL order).
 */
apic_status apic_kk_spectra(apic_plan* plan, int n_tiles, const float* d_intensity,
                            float* d_xdisc, void* stream);

/*
 * Allocation-free Kramers-Kronig stage: the same computation and output as
 * apic_kk_spectra, but its working grids come from one fixed 8 MiB array that
 * the library keeps in device memory from load until process exit, instead of
 * from the plan's workspace. The paper has no counterpart; this entry point
 * exists for callers that cannot allocate device memory when they call: hosts
 * that own all device memory through their own pool or caching allocator and
 * only hand buffers in, and fixed-latency streaming loops where a cudaMalloc
 * (which may synchronise the device) is not acceptable. The call itself makes
 * no cudaMalloc, cudaFree or other allocation; the plan (created earlier)
 * supplies only its read-only geometry tables.
 * Limit: one tile grid of h x w complex values (8 h w bytes) must fit the 8 MiB
 * array, so h w <= 1,048,576 (up to 1024 x 1024); fewer grids fit at once for
 * larger tiles, which lowers parallelism but not correctness. Larger tiles
 * return APIC_EINVAL with a message (apic_last_error).
 * The array comes into being (its module is loaded, 8 MiB of device memory)
 * when the first plan with device memory is created on a device: plan creation
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current, so no call of this entry point is the one that loads it. Each call
 * looks the address up again (cheap once loaded), so the entry point keeps
 * working after cudaDeviceReset once a new plan has been made. All calls share
 * the array: calls that overlap on the GPU (other streams, other host threads)
 * race on it and must be serialised by the caller. Nothing in it needs clearing
 * between calls.
 * Arguments and layouts as apic_kk_spectra; n_tiles is not limited by max_tiles.
 */
apic_status apic_kk_spectra_noalloc(apic_plan* plan, int n_tiles, const float* d_intensity, float* d_xdisc,
                                    void* stream);

/*
 * Aberration solve (Eq. 8-10): phase differences on every overlap S_il,
 * neighbour-difference fit, then least squares on Eq. 10 (FP64 normal
 * equations). d_xdisc as written by apic_kk_spectra; d_zernike [n_tiles][15] out.
 */
apic_status apic_aberration(apic_plan* plan, int n_tiles, const float* d_xdisc,
                            float* d_zernike, void* stream);

/*
 * Correction and stitching: d_spec [n_tiles][n_aperture] complex64 out, the
 * mean of the aberration-corrected spectra at each brightfield aperture point
 * (APIC_TABLE_APERTURE order) and zero on the darkfield-only points.
 */
apic_status apic_stitch(apic_plan* plan, int n_tiles, const float* d_xdisc,
                        const float* d_zernike, float* d_spec, void* stream);

/*
 * Darkfield extension (Eq. 11-13), darkfield images in plan order, each solved
 * by CGLS on C U = b with FFT correlations (FP32 transforms, FP64 scalars and
 * solution accumulation). Updates d_spec in place; ORs APIC_TILE_NOTCONV into
 * d_tile_status (may be NULL) where a solve ended above its tolerance.
 */
apic_status apic_darkfield(apic_plan* plan, int n_tiles, const float* d_intensity,
                           const float* d_zernike, float* d_spec, int32_t* d_tile_status,
                           void* stream);

/* Inverse transform of d_spec onto the (u h) x (u w) grid: d_field out. */
apic_status apic_synthesize(apic_plan* plan, int n_tiles, const float* d_spec, float* d_field,
                            void* stream);

/* Pupil function Circ(k) exp(j phi(k)) (Eq. 1) of each tile: d_pupil [n_tiles][h][w]. */
apic_status apic_pupil(apic_plan* plan, int n_tiles, const float* d_zernike, float* d_pupil,
                       void* stream);

/*
 * Forward model (Eq. 1-2) for synthetic inputs: from objects on the output
 * grid, d_object [n_tiles][u h][u w] complex64 (transmission), and
 * d_zernike [n_tiles][15], write d_intensity [n_tiles][n_bf + n_df][h][w].
 * photons > 0 adds Poisson noise at `photons` per unit intensity from a
 * counter-based generator keyed by (seed, tile, image, pixel).
 */
apic_status apic_simulate(apic_plan* plan, int n_tiles, const float* d_object,
                          const float* d_zernike, float photons, uint64_t seed,
                          float* d_intensity, void* stream);

/*
 * Autotuner (the paper has no counterpart). Times, on the caller's sample
 * d_intensity [n_tiles][n_img][h][w] (1 <= n_tiles <= max_tiles; a full wave
 * of the darkfield grid, e.g. one tile per SM, gives representative numbers),
 * the register-FFT and the shared-memory Stockham variants of the
 * Kramers-Kronig and darkfield stages (best of two runs after a warm-up, CUDA
 * events) and keeps the faster variant of each for the plan's later calls.
 * For 512-pixel tiles the register darkfield kernel is also timed with 1, 2
 * and 4 blocks (a thread-block cluster) per tile, and the fastest kept.
 * h_ms [n_ms] (may be NULL): milliseconds of KK register, KK Stockham,
 * darkfield register (the best cluster size), darkfield Stockham, and the
 * 512-pixel register darkfield kernel with 1, 2, 4 blocks per tile (-1 where
 * a variant does not apply); up to 7 values.
 * Synchronous; uses the plan's workspace, so it must not overlap other calls
 * on the plan.
 */
apic_status apic_plan_autotune(apic_plan* plan, int n_tiles, const float* d_intensity, double* h_ms,
                               int n_ms);

/* ------------------------------------------------------------------------
 * Whole-slide tiling. The paper reconstructs a slide patch by patch
 * (Sec. 2.3, 3.2). No tile is ragged here: windows of the plan's tile size step
 * by `stride` (1..tile) over a slide_h x slide_w camera image, and the last
 * window of each row and column moves inward to end at the slide edge, so one
 * plan serves the whole slide. Consecutive windows split their overlap at its
 * middle: window k owns the slide pixels [oy0, oy1) x [ox0, ox1), and the owned
 * rectangles cover the slide exactly once.
 * Window records: int32 [6] = y0, x0, oy0, ox0, oy1, ox1 (slide pixels).
 * ------------------------------------------------------------------------ */

/* Windows in row-major order into h_windows [capacity][6] (host memory);
 * *n_windows receives their number (h_windows NULL: count only). Host only.
 * Errors: APIC_EINVAL (slide smaller than a tile, stride outside [1, tile],
 * capacity below the count). */
apic_status apic_slide_windows(int slide_h, int slide_w, int tile, int stride, int32_t* h_windows,
                               int capacity, int* n_windows);

/* Cut d_windows [n_tiles][6] (device) out of d_slide [n_img][slide_h][slide_w]
 * float32 into d_intensity [n_tiles][n_img][h][w] (the batch layout). A window
 * that leaves the slide gives a NaN stack, which the reconstruction flags
 * APIC_TILE_BADINPUT. */
apic_status apic_cut_tiles(apic_plan* plan, int n_tiles, const float* d_slide, int slide_h, int slide_w,
                           const int32_t* d_windows, float* d_intensity, void* stream);

/* Write the owned part of each tile's field d_field [n_tiles][u h][u w]
 * complex64 into d_slide_field [u slide_h][u slide_w] complex64; other pixels
 * are left untouched. Each tile keeps its own global phase (the paper's
 * cross-tile registration, Sec. 2.5, is not part of this library). */
apic_status apic_paste_fields(apic_plan* plan, int n_tiles, const float* d_field,
                              const int32_t* d_windows, int slide_h, int slide_w,
                              float* d_slide_field, void* stream);

/* Blend the fields of a slide's whole window grid where windows overlap (the
 * paper reconstructs overlapping patches, Sec. 2.3, 3.2; registration, Sec.
 * 2.5, stays out): n_tiles = n_rows x n_cols windows in apic_slide_windows'
 * row-major order, d_field [n_tiles][u h][u w] complex64, d_windows [n_tiles][6].
 *   d_corr  [n_tiles][2] complex64 out: sum over the overlap with the left /
 *           upper neighbour of f_t conj(f_neighbour) (0 without one);
 *   d_phase [n_tiles] complex64 out: exp(-i phi_t), the tiles' global phases
 *           chained along the grid from these correlations (phi = 0 for the
 *           first window; first row from left neighbours, the rest from upper);
 *   d_slide_field [u slide_h][u slide_w] complex64 out: the sum over covering
 *           windows of w_t exp(-i phi_t) f_t divided by the sum of w_t, with
 *           w_t a product of linear ramps across each overlap (1 elsewhere;
 *           0 where no window covers a pixel).
 * The grid must be a product grid with increasing starts: every window of a
 * row has its row's y0, every window of a column its column's x0 (as
 * apic_slide_windows makes them); other layouts give undefined weights but
 * no access outside the buffers. With u even and d_field, d_slide_field
 * 16-byte aligned the blend moves pixel pairs as 16-byte accesses; otherwise
 * it takes one pixel at a time (same result up to rounding order). Errors:
 * APIC_EINVAL for NULL pointers, n_tiles != n_rows x n_cols, or a slide
 * smaller than a tile. Caller-owned device buffers; asynchronous on `stream`. */
apic_status apic_blend_fields(apic_plan* plan, int n_tiles, const float* d_field, const int32_t* d_windows,
                              int n_rows, int n_cols, int slide_h, int slide_w, float* d_corr, float* d_phase,
                              float* d_slide_field, void* stream);

/* ------------------------------------------------------------------------
 * Learned aberration network. The paper has no counterpart: its aberration
 * estimate is the closed-form solve of Eq. 10 alone. This small CNN predicts
 * the field-dependent Noll coefficients 4..15 of a tile from the magnitudes of
 * its NA-matching intensity spectra and its position, replaces the solve on
 * low-contrast tiles (where Eq. 10 is ill-conditioned) and warm-starts it
 * elsewhere; the closed-form solve stays the fallback and decides, by its
 * residual, which of the two solutions a solved tile keeps.
 *
 * Input features, per tile: feat [64][64][8] float32 (NHWC), channel i =
 *   log(|F(I_i)(kx, ky)| / |F(I_i)(0, 0)| + 1e-4) at [ky + 32][kx + 32],
 *   kx, ky in [-32, 32), F the unnormalised 2-D DFT, I_i the i-th NA-matching
 *   image; uv [2] float32, the tile position on the slide.
 * Layers: conv3x3(pad 1) 8->32, ReLU, maxpool 2 | conv 32->64, ReLU, pool |
 *   conv 64->128, ReLU, pool | conv 128->256, ReLU, global mean | concat uv |
 *   dense 258->256, ReLU | dense 256->12. BF16 weights and layer inputs,
 *   FP32 accumulation, FP32 master weights, gradients and optimizer state.
 * Parameters (apic_net_param_count() = 459244 floats): six row-major
 *   matrices W_l [out_l][taps_l + 1] back to back, bias in the last column;
 *   conv taps ordered (dy, dx, c_in) with dy, dx in 0..2 (offsets -1..1),
 *   dense taps the input features (256 means, then u, v for the first).
 * All device pointers; calls are asynchronous on `stream` unless stated.
 * ------------------------------------------------------------------------ */

/* Floats per parameter vector / per tile of features. */
size_t apic_net_param_count(void);
size_t apic_net_feature_count(void);

/* Network with workspace for batches up to max_batch (1..65536) on the current
 * device; parameters start at zero. Errors: APIC_EINVAL, APIC_ENOMEM, APIC_ECUDA. */
apic_status apic_net_create(int max_batch, apic_net** out);
/* Free the network (synchronises the device first). NULL is a no-op. */
apic_status apic_net_destroy(apic_net* net);

/*
 * Load parameters from a BF16 checkpoint blob in host memory (checkpoint /
 * resume of a trained network; the paper has no network). Layout: the 8 bytes
 * "APICNB16", a little-endian uint32 L, L bytes of a UTF-8 JSON header holding
 * at least "format": "apic-net-bf16" and "count": apic_net_param_count(), then
 * count little-endian BF16 values (the upper 16 bits of IEEE float32) in the
 * apic_net_set_params layout; nothing after them. The values are widened to the
 * network's FP32 master copy (and its BF16 copy), and the AdamW moments zeroed,
 * as apic_net_set_params does. net == NULL only validates the blob. Synchronous.
 * Errors: APIC_EINVAL with a message (short or truncated blob, wrong magic,
 * header, format, count or size), APIC_ECUDA.
 */
apic_status apic_net_load(apic_net* net, const void* h_blob, size_t bytes);

/* Copy parameters from / to host memory (count must be apic_net_param_count());
 * set_params also clears the optimizer moments. Synchronous. */
apic_status apic_net_set_params(apic_net* net, const float* h_params, size_t count);
apic_status apic_net_get_params(const apic_net* net, float* h_params, size_t count);
/* Gradients of the last apic_net_backward, same layout. Synchronous. */
apic_status apic_net_get_grads(const apic_net* net, float* h_grads, size_t count);

/* Forward pass: d_feat [batch][64][64][8] (16-byte aligned), d_uv [batch][2] (NULL: zeros),
 * d_out [batch][15] (Noll 1..3 written as 0; NULL: kept internally). The
 * features must stay valid until the matching apic_net_backward. */
apic_status apic_net_forward(apic_net* net, int batch, const float* d_feat, const float* d_uv,
                             float* d_out, void* stream);
/* Mean squared error of the last forward against d_target [batch][15] (Noll
 * 4..15 used) and its gradient with respect to every parameter. d_loss: one
 * float, or NULL. */
apic_status apic_net_backward(apic_net* net, const float* d_target, float* d_loss, void* stream);
/* AdamW step (bias-corrected moments, decoupled weight decay) with the last
 * gradients; step counts from 1. */
apic_status apic_net_adamw(apic_net* net, float lr, float beta1, float beta2, float eps,
                           float weight_decay, int step, void* stream);
/* Activation of the last forward copied to host float32 (synchronous):
 * which 0..3 the ReLU output of conv layer 0..3 ([batch][H][H][C], H = 64, 32,
 * 16, 8), 4 the dense input [batch][258], 5 the hidden layer [batch][256], 6 the
 * outputs [batch][12]. count must match. */
apic_status apic_net_activation(const apic_net* net, int which, float* h_out, size_t count);

/* Network input features of n_tiles stacks (the plan's first 8 images, which
 * must be its 8 NA-matching images): d_feat [n_tiles][64][64][8]. Tiles of 64,
 * 128 or 256 pixels. */
apic_status apic_features(apic_plan* plan, int n_tiles, const float* d_intensity, float* d_feat,
                          void* stream);

/* Learned-assisted reconstruction modes. */
#define APIC_NET_WARM     1   /* solved tiles also refine from the network's coefficients and
                                 keep the solution with the smaller wrapped residual        */
#define APIC_NET_REPLACE  2   /* tiles below bg_contrast take the network's coefficients and
                                 are reconstructed with them (APIC_TILE_LEARNED)             */

/*
 * apic_reconstruct_batch with the network: features and network forward per
 * chunk, then the stages as there, with the aberration stage per `mode`.
 * d_uv [n_tiles][2] tile positions. With APIC_NET_REPLACE low-contrast tiles
 * are never skipped. Same buffers and errors as apic_reconstruct_batch. The
 * first call on a plan allocates its feature and coefficient buffers
 * (max_tiles tiles), so make one call before capturing this one in a CUDA
 * graph; apic_reconstruct_batch allocates nothing after plan creation.
 */
apic_status apic_reconstruct_learned(apic_plan* plan, apic_net* net, int mode, int n_tiles,
                                     const float* d_intensity, const float* d_uv, float* d_field,
                                     float* d_zernike, float* d_pupil, int32_t* d_tile_status,
                                     void* stream);

#ifdef __cplusplus
}
#endif
#endif /* APIC_H */
