// plan.cpp - host-side geometry of one tile-size class (WSI-APIC, Sec. 2.2-2.3).
//
// Readings of the paper used here (the paper states the continuous method):
//  * Pupil: ellipse (kx/Rx)^2 + (ky/Ry)^2 <= 1 + 1e-9 on integer frequencies,
//    Rx = NA w dx / lambda, Ry = NA h dx / lambda (Circ_NA of Eq. 1).
//  * NA-matching LEDs are snapped to the nearest grid point inside the pupil
//    whose shifted pupil keeps every point other than DC on the negative side
//    of the line k . k_i = 0 - the DC-on-the-edge condition that Eq. 5
//    relies on. Darkfield LEDs snap to floor(p + 0.5).
//  * Overlap sets S_il (Eq. 8) for pairs i < l; rows of D (Eq. 10) in the
//    Zernike basis j = 4..15, with neighbour links for the wrap-free
//    difference fit.
//  * Darkfield images in order of increasing |k|, then angle; unknown U and
//    known P split of each disc, Q = (U - P) minus (P - U) and (U - U); an
//    image is used only if M >= N and N <= 0.42 |D| (Sec. 4).
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <tuple>

#include "zernike.h"

namespace apic {

namespace {
struct DFGrid {
    int mx, my;
    double col_cost;   // relative cost of one column of my points (paired when my <= 128)
};
const DFGrid kDFGrids[] = {{192, 192, 2.0}, {192, 144, 1.68}, {192, 128, 1.13}, {192, 96, 1.0},
                           {160, 128, 1.13}, {160, 96, 1.0},  {144, 144, 1.68}};
}  // namespace

// Wide kernel (512-point camera grid): rows of 288 or 320 points, columns of 192,
// 256, 288 or 320 points (a column of more than 256 points costs two DFT_16 steps
// per lane instead of one).
const DFGrid kDFWideGrids[] = {{288, 192, 1.0}, {288, 256, 1.12}, {288, 288, 1.62},
                               {320, 192, 1.0}, {320, 256, 1.12}, {320, 288, 1.62}, {320, 320, 1.65}};

bool df_grid_supported(int mx, int my) {
    for (const DFGrid& g : kDFGrids)
        if (g.mx == mx && g.my == my) return true;
    return false;
}

bool df_wide_grid_supported(int mx, int my) {
    for (const DFGrid& g : kDFWideGrids)
        if (g.mx == mx && g.my == my) return true;
    return false;
}

// Along each axis the correlations of Eq. 13 are exact on a circular grid of L
// points when C u (U with P, read on Q) has no q - p - k (q in U, p in P, k in Q)
// that is a nonzero multiple of L and C^H r (Q with P, read on U) no such
// k + p - q, and every band fits: the least such L along the solve frame's rows
// (nx) and columns (ny).
void df_grid_needs(const DarkfieldHost& d, int& nx, int& ny) {
    auto need = [](const std::vector<int>& U, const std::vector<int>& Pv, const std::vector<int>& Q) {
        auto mm = [](const std::vector<int>& v) { return std::minmax_element(v.begin(), v.end()); };
        const auto u = mm(U), pp = mm(Pv), q = mm(Q);
        const int u0 = *u.first, u1 = *u.second, p0 = *pp.first, p1 = *pp.second, q0 = *q.first, q1 = *q.second;
        const int need_c = std::max(std::abs(u0 - p1 - q1), std::abs(u1 - p0 - q0)) + 1;
        const int need_ch = std::max(std::abs(q0 + p0 - u1), std::abs(q1 + p1 - u0)) + 1;
        return std::max({need_c, need_ch, u1 - u0 + 1, p1 - p0 + 1, q1 - q0 + 1});
    };
    nx = ny = 0;
    if (d.U_x.empty() || d.P_x.empty() || d.Q_x.empty()) return;
    const bool tr = d.solve_tr != 0;         // solve frame: rows run along x' = (tr ? y : x)
    nx = tr ? need(d.U_y, d.P_y, d.Q_y) : need(d.U_x, d.P_x, d.Q_x);
    ny = tr ? need(d.U_x, d.P_x, d.Q_x) : need(d.U_y, d.P_y, d.Q_y);
}

// Frame and grid of the register-kernel solve of one darkfield image (an
// implementation choice; the problem of Eq. 13 is unchanged):
// - an image whose lag set Q is narrower along x than along y is solved
//   transposed (x <-> y in every set and in the image), so the row bands the
//   darkfield passes walk are the shorter ones;
// - of the supported (row, column) grids on the 192-point register grid, the
//   exact one (df_grid_needs) with the least estimated work per iteration
//   (columns x relative cost of a column) is used. Other register grids use
//   mr x mr.
// - on the wide kernel's 512-point grid (512-pixel tiles) the row and column grids
//   come from kDFWideGrids alone; returns false when none is exact for the image.
static bool solve_grid(DarkfieldHost& d, int mr) {
    auto extent = [](const std::vector<int>& v) {
        return v.empty() ? 0 : *std::max_element(v.begin(), v.end()) - *std::min_element(v.begin(), v.end()) + 1;
    };
    d.solve_tr = extent(d.Q_x) < extent(d.Q_y) ? 1 : 0;
    d.solve_mx = d.solve_my = mr;
    if ((mr != 192 && mr != 512) || d.U_x.empty() || d.P_x.empty() || d.Q_x.empty()) return true;
    int nx = 0, ny = 0;
    df_grid_needs(d, nx, ny);
    double best = 1e300;
    bool found = mr != 512;
    for (const DFGrid& g : (mr == 512 ? kDFWideGrids : kDFGrids))
        if (g.mx >= nx && g.my >= ny && g.mx * g.col_cost < best) {
            best = g.mx * g.col_cost;
            d.solve_mx = g.mx;
            d.solve_my = g.my;
            found = true;
        }
    return found;
}
namespace {

constexpr double kPupilTol = 1e-9;
constexpr double kUnknownMax = 0.42;

struct Geo {
    int h, w;
    double Rx, Ry;
    bool in_pupil(long kx, long ky) const {
        const double x = (double)kx, y = (double)ky;
        return (x * x) / (Rx * Rx) + (y * y) / (Ry * Ry) <= 1.0 + kPupilTol;
    }
};

// No grid point K != 0 of the pupil shifted by -k lies on the closed side
// K . k >= 0 (physical dot product); such a point needs ||K||^2 <= slack.
bool edge_clean(const Geo& g, int kx, int ky) {
    const double slack =
        1.0 + kPupilTol - (((double)((long)kx * kx)) / (g.Rx * g.Rx) + ((double)((long)ky * ky)) / (g.Ry * g.Ry));
    if (slack < 0) return false;
    const int ax = (int)std::floor(g.Rx * std::sqrt(slack)) + 1;
    const int ay = (int)std::floor(g.Ry * std::sqrt(slack)) + 1;
    const long hh = (long)g.h * g.h, ww = (long)g.w * g.w;
    for (int qy = -ay; qy <= ay; ++qy)
        for (int qx = -ax; qx <= ax; ++qx) {
            if (qx == 0 && qy == 0) continue;
            const long dot = (long)qx * kx * hh + (long)qy * ky * ww;
            if (dot < 0) continue;
            if (g.in_pupil(qx + kx, qy + ky)) return false;
        }
    return true;
}

void cholesky12(const double* G, double* L) {
    for (int i = 0; i < 144; ++i) L[i] = 0;
    for (int j = 0; j < 12; ++j) {
        double d = G[j * 12 + j];
        for (int k = 0; k < j; ++k) d -= L[j * 12 + k] * L[j * 12 + k];
        d = std::sqrt(std::max(d, 1e-300));
        L[j * 12 + j] = d;
        for (int i = j + 1; i < 12; ++i) {
            double s = G[i * 12 + j];
            for (int k = 0; k < j; ++k) s -= L[i * 12 + k] * L[j * 12 + k];
            L[i * 12 + j] = s / d;
        }
    }
}

struct BoolGrid {  // dense boolean map over [-half, half]^2
    int half = 0, size = 0;
    std::vector<uint8_t> v;
    explicit BoolGrid(int hf) : half(hf), size(2 * hf + 1), v((size_t)size * size, 0) {}
    uint8_t& at(int x, int y) { return v[(size_t)(y + half) * size + (x + half)]; }
    bool get(int x, int y) const {
        if (x < -half || x > half || y < -half || y > half) return false;
        return v[(size_t)(y + half) * size + (x + half)] != 0;
    }
};

// A point set ordered by (y, x) as runs of consecutive x on each row: (y, x0, x1), inclusive.
struct Run {
    int y, x0, x1;
};

std::vector<Run> runs_of(const std::vector<int>& xs, const std::vector<int>& ys) {
    std::vector<Run> r;
    for (size_t i = 0; i < xs.size(); ++i) {
        if (!r.empty() && r.back().y == ys[i] && r.back().x1 + 1 == xs[i])
            r.back().x1 = xs[i];
        else
            r.push_back({ys[i], xs[i], xs[i]});
    }
    return r;
}

// Marks {a - b : a in A, b in B} into out. The difference of the runs [a0, a1] on row ya
// and [b0, b1] on row yb is the run [a0 - b1, a1 - b0] on row ya - yb, so each pair of
// runs costs one increment and one decrement in a per-row counter; a prefix sum over each
// row then marks every point that some pair covers.
void mark_difference(const std::vector<Run>& A, const std::vector<Run>& B, BoolGrid& out) {
    const int half = out.half, size = out.size;
    std::vector<int> cnt((size_t)size * (size + 1), 0);
    for (const Run& a : A)
        for (const Run& b : B) {
            int* row = cnt.data() + (size_t)(a.y - b.y + half) * (size + 1);
            row[a.x0 - b.x1 + half] += 1;
            row[a.x1 - b.x0 + half + 1] -= 1;
        }
    for (int y = 0; y < size; ++y) {
        const int* row = cnt.data() + (size_t)y * (size + 1);
        int c = 0;
        for (int x = 0; x < size; ++x) {
            c += row[x];
            if (c > 0) out.v[(size_t)y * size + x] = 1;
        }
    }
}

}  // namespace

int HostPlan::pupil_index(int kx, int ky) const {
    if (kx < -pup_ax || kx > pup_ax || ky < -pup_ay || ky > pup_ay) return -1;
    return pup_lut[(size_t)(ky + pup_ay) * (2 * pup_ax + 1) + (kx + pup_ax)];
}

std::string build_host_plan(const GeomParams& p, HostPlan& P) {
    P = HostPlan();
    P.h = p.h;
    P.w = p.w;
    P.up = p.up;
    P.H = p.up * p.h;
    P.W = p.up * p.w;
    P.n_bf = p.n_bf;
    P.n_df = p.n_df;
    P.Rx = (p.na * (double)p.w * p.dx) / p.wl;
    P.Ry = (p.na * (double)p.h * p.dx) / p.wl;
    const Geo g{p.h, p.w, P.Rx, P.Ry};
    const int n_img = p.n_bf + p.n_df;

    // ---- snap the illumination
    const int win = 2 + (int)std::floor(0.2 * std::max(P.Rx, P.Ry));
    for (int idx = 0; idx < n_img; ++idx) {
        const double px = p.kx[idx] * (double)p.w * p.dx;
        const double py = p.ky[idx] * (double)p.h * p.dx;
        if (idx < p.n_bf) {
            bool found = false;
            double bd = 0;
            int bx = 0, by = 0;
            const int fx = (int)std::floor(px), fy = (int)std::floor(py);
            for (int cy = fy - win; cy <= fy + win; ++cy)
                for (int cx = fx - win; cx <= fx + win; ++cx) {
                    if (!g.in_pupil(cx, cy)) continue;
                    const double d2 = (cx - px) * (cx - px) + (cy - py) * (cy - py);
                    if (found && std::make_tuple(d2, cy, cx) >= std::make_tuple(bd, by, bx)) continue;
                    if (!edge_clean(g, cx, cy)) continue;
                    found = true;
                    bd = d2;
                    bx = cx;
                    by = cy;
                }
            if (!found) return "NA-matching LED " + std::to_string(idx) + " has no admissible grid point";
            P.led_x.push_back(bx);
            P.led_y.push_back(by);
        } else {
            P.led_x.push_back((int)std::floor(px + 0.5));
            P.led_y.push_back((int)std::floor(py + 0.5));
        }
    }

    // ---- pupil points, ordered by (ky, kx)
    P.pup_ax = (int)std::ceil(P.Rx) + 1;
    P.pup_ay = (int)std::ceil(P.Ry) + 1;
    P.pup_lut.assign((size_t)(2 * P.pup_ax + 1) * (2 * P.pup_ay + 1), -1);
    for (int ky = -P.pup_ay; ky <= P.pup_ay; ++ky)
        for (int kx = -P.pup_ax; kx <= P.pup_ax; ++kx)
            if (g.in_pupil(kx, ky)) {
                P.pup_lut[(size_t)(ky + P.pup_ay) * (2 * P.pup_ax + 1) + (kx + P.pup_ax)] = (int)P.pup_x.size();
                P.pup_x.push_back(kx);
                P.pup_y.push_back(ky);
            }
    const int npup = (int)P.pup_x.size();
    int rint = 0;
    for (int i = 0; i < npup; ++i) rint = std::max(rint, std::max(std::abs(P.pup_x[i]), std::abs(P.pup_y[i])));
    for (int i = 0; i < p.n_bf; ++i) {
        const int q = P.pupil_index(P.led_x[i], P.led_y[i]);
        if (q < 0) return "NA-matching LED outside the pupil";
        P.led_pup.push_back(q);
    }

    // ---- known region: object-frequency grid covering the output spectrum
    const int khalf = std::max(P.H, P.W);
    BoolGrid known(khalf);
    for (int i = 0; i < p.n_bf; ++i)
        for (int q = 0; q < npup; ++q) known.at(P.pup_x[q] - P.led_x[i], P.pup_y[q] - P.led_y[i]) = 1;

    // ---- darkfield order: |k|^2, then angle, then index
    std::vector<std::tuple<long, double, int>> order;
    for (int j = 0; j < p.n_df; ++j) {
        const int x = P.led_x[p.n_bf + j], y = P.led_y[p.n_bf + j];
        order.emplace_back((long)x * x + (long)y * y, std::atan2((double)y, (double)x), j);
    }
    std::sort(order.begin(), order.end());

    for (auto& o : order) {
        const int j = std::get<2>(o);
        DarkfieldHost d;
        d.led = p.n_bf + j;
        d.kx = P.led_x[d.led];
        d.ky = P.led_y[d.led];
        d.n_disc = npup;
        int dmax = 0;
        for (int q = 0; q < npup; ++q) {
            const int Kx = P.pup_x[q] - d.kx, Ky = P.pup_y[q] - d.ky;   // object frequency
            dmax = std::max(dmax, std::max(std::abs(Kx), std::abs(Ky)));
            if (std::abs(Kx) > khalf || std::abs(Ky) > khalf) return "darkfield disc outside the object grid";
            if (known.get(Kx, Ky)) {
                d.P_x.push_back(P.pup_x[q]);
                d.P_y.push_back(P.pup_y[q]);
                d.P_pup.push_back(q);
            } else {
                d.U_x.push_back(P.pup_x[q]);
                d.U_y.push_back(P.pup_y[q]);
                d.U_pup.push_back(q);
            }
        }
        // Q from the set differences (lags are frame independent); P - U is U - P mirrored
        const int half = 2 * dmax + 1;
        BoolGrid up(half), uu(half);
        const std::vector<Run> Ur = runs_of(d.U_x, d.U_y), Pr = runs_of(d.P_x, d.P_y);
        mark_difference(Ur, Pr, up);
        mark_difference(Ur, Ur, uu);
        for (int y = -half; y <= half; ++y)
            for (int x = -half; x <= half; ++x)
                if (up.get(x, y) && !up.get(-x, -y) && !uu.get(x, y)) {
                    d.Q_x.push_back(x);
                    d.Q_y.push_back(y);
                }
        const size_t N = d.U_x.size(), M = d.Q_x.size();
        d.used = N > 0 && M >= N && (double)N <= kUnknownMax * (double)npup;
        if (d.used)
            for (size_t u = 0; u < N; ++u) known.at(d.U_x[u] - d.kx, d.U_y[u] - d.ky) = 1;
        P.df.push_back(std::move(d));
    }

    // ---- synthetic aperture, ordered by (ky, kx)
    std::vector<int> ap_lut(known.v.size(), -1);
    for (int y = -khalf; y <= khalf; ++y)
        for (int x = -khalf; x <= khalf; ++x)
            if (known.get(x, y)) {
                if (std::abs(x) >= P.W / 2 || std::abs(y) >= P.H / 2)
                    return "spectrum support exceeds the upsampled grid";
                ap_lut[(size_t)(y + khalf) * known.size + (x + khalf)] = (int)P.ap_x.size();
                P.ap_x.push_back(x);
                P.ap_y.push_back(y);
            }
    auto ap_index = [&](int x, int y) { return ap_lut[(size_t)(y + khalf) * known.size + (x + khalf)]; };
    const int nap = (int)P.ap_x.size();

    // ---- brightfield stitch lists
    std::vector<std::vector<std::pair<int, int>>> lists(nap);
    for (int i = 0; i < p.n_bf; ++i)
        for (int q = 0; q < npup; ++q) lists[ap_index(P.pup_x[q] - P.led_x[i], P.pup_y[q] - P.led_y[i])].push_back({i, q});
    P.ap_bf.assign(nap, 0);
    P.st_ptr.push_back(0);
    for (int a = 0; a < nap; ++a) {
        for (auto& e : lists[a]) {
            P.st_img.push_back(e.first);
            P.st_pup.push_back(e.second);
        }
        P.ap_bf[a] = lists[a].empty() ? 0 : 1;
        P.st_ptr.push_back((int)P.st_img.size());
    }
    for (auto& d : P.df) {
        for (size_t u = 0; u < d.U_x.size(); ++u) d.U_ap.push_back(ap_index(d.U_x[u] - d.kx, d.U_y[u] - d.ky));
        for (size_t q = 0; q < d.P_x.size(); ++q) d.P_ap.push_back(ap_index(d.P_x[q] - d.kx, d.P_y[q] - d.ky));
    }

    // ---- aberration rows (Eq. 10)
    double Gv[144] = {0}, Gg[144] = {0};
    std::vector<double> Ad;   // double copy for the normal matrices
    for (int i = 0; i < p.n_bf; ++i)
        for (int l = i + 1; l < p.n_bf; ++l) {
            double zi[12], zl[12];
            zernike_4_15<double>(P.led_x[i] / P.Rx, P.led_y[i] / P.Ry, zi);
            zernike_4_15<double>(P.led_x[l] / P.Rx, P.led_y[l] / P.Ry, zl);
            const size_t first = P.row_i.size();
            std::map<std::pair<int, int>, int> where;
            for (int q = 0; q < npup; ++q) {
                const int Kx = P.pup_x[q] - P.led_x[i], Ky = P.pup_y[q] - P.led_y[i];
                const int ql = P.pupil_index(Kx + P.led_x[l], Ky + P.led_y[l]);
                if (ql < 0) continue;
                double a[12], b[12];
                zernike_4_15<double>((Kx + P.led_x[i]) / P.Rx, (Ky + P.led_y[i]) / P.Ry, a);
                zernike_4_15<double>((Kx + P.led_x[l]) / P.Rx, (Ky + P.led_y[l]) / P.Ry, b);
                where[{Kx, Ky}] = (int)P.row_i.size();
                P.row_i.push_back(i);
                P.row_l.push_back(l);
                P.row_pi.push_back(q);
                P.row_pl.push_back(ql);
                for (int z = 0; z < 12; ++z) {
                    const double v = a[z] - b[z] - zi[z] + zl[z];
                    Ad.push_back(v);
                    P.row_A.push_back((float)v);
                }
            }
            for (size_t r = first; r < P.row_i.size(); ++r) {
                const int Kx = P.pup_x[P.row_pi[r]] - P.led_x[i], Ky = P.pup_y[P.row_pi[r]] - P.led_y[i];
                auto fx = where.find({Kx + 1, Ky});
                auto fy = where.find({Kx, Ky + 1});
                P.row_nx.push_back(fx == where.end() ? -1 : fx->second);
                P.row_ny.push_back(fy == where.end() ? -1 : fy->second);
            }
        }
    const size_t nrows = P.row_i.size();
    if (nrows < 12) return "too few overlap rows for the aberration solve";
    for (size_t r = 0; r < nrows; ++r) {
        const double* a = &Ad[r * 12];
        for (int u = 0; u < 12; ++u)
            for (int v = 0; v < 12; ++v) Gv[u * 12 + v] += a[u] * a[v];
        for (int dir = 0; dir < 2; ++dir) {
            const int r2 = dir == 0 ? P.row_nx[r] : P.row_ny[r];
            if (r2 < 0) continue;
            const double* b = &Ad[(size_t)r2 * 12];
            for (int u = 0; u < 12; ++u)
                for (int v = 0; v < 12; ++v) Gg[u * 12 + v] += (b[u] - a[u]) * (b[v] - a[v]);
        }
    }
    cholesky12(Gv, P.Lval);
    cholesky12(Gg, P.Lgrad);

    // ---- correlation grid: alias-free for lags up to 2 rint (m >= 4 rint + 1)
    P.m = 16;
    while (P.m < 4 * rint + 1) P.m *= 2;
    for (int B : {4, 6, 8, 12, 16})
        if (16 * B >= 4 * rint + 1) {
            P.mr = 16 * B;
            break;
        }
    // 512-pixel tiles: the wide kernel (P * P on the camera grid, per-image CG grids)
    if (P.mr == 0 && p.h == 512 && p.w == 512 && 4 * rint + 1 <= 512) P.mr = 512;
    bool grids_ok = true;
    for (auto& d : P.df)
        if (d.used) grids_ok = solve_grid(d, P.mr) && grids_ok;
    if (!grids_ok) {     // some image needs a longer grid than the wide kernel has
        P.mr = 0;
        for (auto& d : P.df) d.solve_mx = d.solve_my = 0;
    }
    for (auto& d : P.df)
        for (size_t q = 0; q < d.Q_x.size(); ++q)
            if (2 * std::abs(d.Q_x[q]) >= p.w || 2 * std::abs(d.Q_y[q]) >= p.h)
                return "darkfield lags exceed the camera grid";
    return "";
}

}  // namespace apic
