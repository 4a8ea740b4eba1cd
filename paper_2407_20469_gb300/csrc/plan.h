// plan.h - host-side geometry of one tile-size class: snapped illumination,
// pupil points, synthetic aperture, overlap rows of the aberration system and
// the darkfield index sets. Built once per plan; the kernels index into the
// tables it produces.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace apic {

struct GeomParams {
    int h, w, up, n_bf, n_df;
    double na, wl, dx;                  // float32 inputs widened to double
    std::vector<double> kx, ky;         // cycles/um, float32 inputs widened
};

// One darkfield image: index sets of Eq. 11-13 in camera coordinates
// c = K + k_j (the pupil frame), each sorted by (y, x).
struct DarkfieldHost {
    int led;                  // index into the LED list (n_bf + j)
    int kx, ky;               // snapped wave-vector
    bool used;                // false: skipped (M < N or N > 0.42 |D|, Sec. 4)
    int n_disc;
    std::vector<int> U_x, U_y, U_pup, U_ap;   // unknown points, their pupil and aperture index
    std::vector<int> P_x, P_y, P_pup, P_ap;   // known points
    std::vector<int> Q_x, Q_y;                // equation lags (k of Eq. 13)
    // frame and grid of the register-kernel solve (used images): solved transposed, row grid
    // points, column grid points (mr x mr unless a shorter supported grid is exact; 0 without
    // the register grid)
    int solve_tr = 0, solve_mx = 0, solve_my = 0;
};

struct HostPlan {
    int h = 0, w = 0, H = 0, W = 0, up = 0, n_bf = 0, n_df = 0;
    double Rx = 0, Ry = 0;
    std::vector<int> led_x, led_y;            // snapped (kx, ky), all LEDs
    // pupil points (Circ_NA of Eq. 1), ordered by (ky, kx)
    std::vector<int> pup_x, pup_y;
    int pup_ax = 0, pup_ay = 0;               // half extents of the lookup box
    std::vector<int> pup_lut;                 // (2ay+1)(2ax+1) -> index or -1
    std::vector<int> led_pup;                 // NA-matching LED -> pupil index of k_i
    // synthetic aperture (object frequencies), ordered by (ky, kx)
    std::vector<int> ap_x, ap_y;
    std::vector<uint8_t> ap_bf;               // 1 if covered by a brightfield disc
    // brightfield stitch lists: aperture point -> (image, pupil index) entries
    std::vector<int> st_ptr, st_img, st_pup;
    // aberration rows (Eq. 10), pairs i < l
    std::vector<int> row_i, row_l, row_pi, row_pl, row_nx, row_ny;
    std::vector<float> row_A;                 // [rows][12]
    double Lval[144] = {0}, Lgrad[144] = {0}; // Cholesky factors (lower, row-major)
    // darkfield images in processing order (increasing |k|, then angle)
    std::vector<DarkfieldHost> df;
    int m = 0;                                // grid of the darkfield correlations (power of two)
    int mr = 0;                               // register-FFT grid 16 B (B in 4, 6, 8, 12, 16; 512 for the
                                              // wide kernel of 512-pixel tiles), 0 if none

    int pupil_index(int kx, int ky) const;
};

// Builds the plan; returns an empty string on success, else the reason.
std::string build_host_plan(const GeomParams& p, HostPlan& out);
// Supported (row, column) grids of the register darkfield solve on the 192-point grid,
// and of the wide kernel's solve (512-pixel tiles).
bool df_grid_supported(int mx, int my);
bool df_wide_grid_supported(int mx, int my);
// Least alias-free grid lengths of a used darkfield image along its solve frame's rows and columns.
void df_grid_needs(const DarkfieldHost& d, int& nx, int& ny);

}  // namespace apic
