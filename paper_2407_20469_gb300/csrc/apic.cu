// apic.cu - C interface of the library (include/apic.h): plan creation, table
// upload, workspace, stage entry points and the batched reconstruction.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/apic.h"
#include "internal.cuh"
#include "passes.cuh"
#include "plan.h"

using namespace apic;

namespace {

thread_local std::string g_last_error;

apic_status fail(apic_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

apic_status cuda_fail(cudaError_t e, const char* where) {
    return fail(APIC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define APIC_TRY_CUDA(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return cuda_fail(_e, #expr);   \
    } while (0)

// Packs host vectors into one device allocation.
struct Arena {
    std::vector<char> host;
    template <typename T>
    size_t add(const T* p, size_t count) {
        size_t off = (host.size() + 255) & ~(size_t)255;
        host.resize(off + count * sizeof(T));
        if (count) std::memcpy(host.data() + off, p, count * sizeof(T));
        return off;
    }
    template <typename T>
    size_t add(const std::vector<T>& v) {
        return add(v.data(), v.size());
    }
};

std::vector<int> rowptr_of(const std::vector<int>& ys, int y0, int y1) {
    std::vector<int> rp(std::max(0, y1 - y0 + 1) + 1, 0);
    for (int y : ys) rp[y - y0 + 1]++;
    for (size_t i = 1; i < rp.size(); ++i) rp[i] += rp[i - 1];
    return rp;
}

std::vector<float2> twiddles(int N) {
    std::vector<float2> t(N);
    for (int k = 0; k < N; ++k) {
        const double a = -2.0 * M_PI * (double)k / (double)N;
        t[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    return t;
}

bool pow2(int n) { return n >= 16 && (n & (n - 1)) == 0; }

}  // namespace

struct apic_plan {
    apic_params params;
    HostPlan host;
    DevPlan dev;
    Launch L;
    int device = 0, sms = 0;
    int max_tiles = 0, df_iters = 40, ab_passes = 2;
    float df_tol = 3e-4f, bg_thresh2 = 4e-4f, bg_c2 = 4e-4f;
    void* d_tables = nullptr;
    // workspace
    float2* xdisc = nullptr;
    float* zern = nullptr;
    float* phi = nullptr;
    float2* spec = nullptr;
    int32_t* status = nullptr;
    float* c2 = nullptr;
    float2* kk_scratch = nullptr;
    float* beta_scratch = nullptr;
    void* df_scratch = nullptr;
    size_t df_per_block = 0;
    float2* sim_scratch = nullptr;
    size_t sim_bytes = 0;
    std::vector<void*> allocs;
    bool host_only = false;
    bool use_reg = false;        // register-FFT darkfield kernel
    size_t smem_dfr = 0;
    int grid_dfr = 0;            // tile slots of the register darkfield kernel (blocks, or clusters of
                                 // df_cluster blocks for the wide kernel)
    int df_cluster = 1;          // blocks per tile of the wide darkfield kernel
    int dfw_slots[3] = {0, 0, 0};   // wide kernel: tile slots with 1, 2, 4 blocks per tile
    int df_slots_alloc = 0;      // tile slots of each half of the darkfield scratch
    // host-buffer pipeline (apic_reconstruct_host), created on first use
    struct HostIO {
        bool ready = false;
        int chunk = 0;           // tiles per chunk of the chunked order (buffer sets 0 and 1)
        int one = 0;             // tiles buffer set 0 holds: calls of up to `one` tiles take the one-chunk order
        int cap[2] = {0, 0};     // tiles each buffer set holds (0: not allocated)
        cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
        cudaEvent_t in_done[2] = {}, comp_done[2] = {}, out_done[2] = {};
        cudaEvent_t in_tail = nullptr, early = nullptr;   // one-chunk order
        cudaEvent_t part[16] = {};                         // one-chunk order: the full waves' inputs in parts
        cudaEvent_t rdone[32] = {};                        // one-chunk order: fields of the first group's rounds
        cudaEvent_t ml_done = nullptr;                     // one-chunk order: fields of the second group's early rounds
        float* d_in[2] = {};
        float* d_field[2] = {};
        float* d_zern[2] = {};
        int32_t* d_status[2] = {};
    } io;
    bool kkr_ok = false, dfr_ok = false;   // register kernels available for this geometry
    bool use_kkr = false;        // register-FFT Kramers-Kronig kernel
    size_t smem_kkr = 0;
    int grid_kkr = 0;
    // second stream for the last partial darkfield wave of a batch (see reconstruct)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_tail = nullptr, ev_pre = nullptr, ev_mbe = nullptr;
    // inputs arriving per group of darkfield rounds (host pipeline): the groups' earlier
    // stages on a stream of their own, one event per group
    cudaStream_t prep = nullptr;
    cudaEvent_t ev_prep[16] = {};
    float* feat = nullptr;                       // learned path: features, network coefficients
    float* c_net = nullptr;
    unsigned long long* d_counters = nullptr;   // kCounters: [1] CG iterations, [2] solves, [4 + i] per image
    int* d_work = nullptr;                       // tile counters of the darkfield launches: [0] caller's stream,
                                                 // [1] the second stream
    long long launches = 0;                      // kernel launches issued
    // stage timing: ring of kTimingSlots calls x kStages x {start, stop}
    bool timing = false;
    std::vector<cudaEvent_t> events;
    int t_next = 0, t_used = 0;
    static constexpr int kStages = 7, kTimingSlots = 1024;
};

namespace {

apic_status dmalloc(apic_plan* p, void** ptr, size_t bytes) {
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(APIC_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed");
    }
    p->allocs.push_back(*ptr);
    return APIC_OK;
}

apic_status upload(apic_plan* plan) {
    const HostPlan& H = plan->host;
    DevPlan& D = plan->dev;
    Arena A;
    D = DevPlan();
    D.h = H.h;
    D.w = H.w;
    D.H = H.H;
    D.W = H.W;
    D.n_bf = H.n_bf;
    D.n_df = H.n_df;
    D.n_img = H.n_bf + H.n_df;
    D.npup = (int)H.pup_x.size();
    D.nap = (int)H.ap_x.size();
    D.nrows = (int)H.row_i.size();
    D.m = H.m;
    D.Rx = (float)H.Rx;
    D.Ry = (float)H.Ry;
    D.pup_ax = H.pup_ax;
    D.pup_ay = H.pup_ay;

    const size_t o_pupx = A.add(H.pup_x), o_pupy = A.add(H.pup_y), o_lut = A.add(H.pup_lut);
    const size_t o_puprp = A.add(rowptr_of(H.pup_y, -H.pup_ay, H.pup_ay));
    const size_t o_ledx = A.add(H.led_x), o_ledy = A.add(H.led_y), o_ledp = A.add(H.led_pup);
    std::vector<int> il(H.row_i.size());
    for (size_t r = 0; r < il.size(); ++r) il[r] = H.row_i[r] | (H.row_l[r] << 16);
    const size_t o_il = A.add(il), o_pi = A.add(H.row_pi), o_pl = A.add(H.row_pl);
    const size_t o_nx = A.add(H.row_nx), o_ny = A.add(H.row_ny), o_A = A.add(H.row_A);
    const size_t o_Lv = A.add(H.Lval, 144), o_Lg = A.add(H.Lgrad, 144);
    const size_t o_apx = A.add(H.ap_x), o_apy = A.add(H.ap_y), o_apbf = A.add(H.ap_bf);
    const size_t o_stp = A.add(H.st_ptr), o_sti = A.add(H.st_img), o_stq = A.add(H.st_pup);
    int ay0 = 0, ay1 = -1;
    if (!H.ap_y.empty()) {
        ay0 = H.ap_y.front();
        ay1 = H.ap_y.back();
    }
    D.ap_y0 = ay0;
    D.ap_y1 = ay1;
    const size_t o_aprp = A.add(rowptr_of(H.ap_y, ay0, ay1));
    // the aperture list in (x, y) order, by columns ap_x0..ap_x1 (register synthesis)
    int ax0 = 0, ax1 = -1;
    if (!H.ap_x.empty()) {
        ax0 = *std::min_element(H.ap_x.begin(), H.ap_x.end());
        ax1 = *std::max_element(H.ap_x.begin(), H.ap_x.end());
    }
    const std::vector<int> colptr = rowptr_of(H.ap_x, ax0, ax1);
    std::vector<int> cole(H.ap_x.size()), fillp(colptr.begin(), colptr.end() - 1);
    for (size_t q = 0; q < H.ap_x.size(); ++q) cole[fillp[H.ap_x[q] - ax0]++] = (int)q;
    D.ap_x0 = ax0;
    D.ap_x1 = ax1;
    const size_t o_apcp = A.add(colptr), o_apce = A.add(cole);

    // darkfield tables
    std::vector<DevDF> dfs;
    std::vector<int> ux, uy, up, ua, px, py, pp, pa, qx, qy, rp;
    std::vector<unsigned> qmask;
    int maxN = 1, maxM = 1, band_u = 1, band_p = 1, band_q = 1, max_mx = 16, max_mxy = 256;
    const int mr = H.mr;
    for (const auto& d : H.df) {
        if (!d.used) continue;
        DevDF e{};
        e.led = d.led;
        e.kx = d.kx;
        e.ky = d.ky;
        e.N = (int)d.U_x.size();
        e.M = (int)d.Q_x.size();
        e.NP = (int)d.P_x.size();
        // Solve frame and grid chosen with the host plan (x <-> y swapped in every
        // set and in the image when d.solve_tr); points are re-sorted by their new rows.
        const bool tr = d.solve_tr != 0;
        e.tr = tr ? 1 : 0;
        struct Set {
            std::vector<int> x, y, pup, ap;
        };
        auto frame = [&](const std::vector<int>& xs, const std::vector<int>& ys, const std::vector<int>* pup,
                         const std::vector<int>* ap) {
            const std::vector<int>& fx = tr ? ys : xs;
            const std::vector<int>& fy = tr ? xs : ys;
            std::vector<size_t> idx(xs.size());
            for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
            if (tr)
                std::stable_sort(idx.begin(), idx.end(), [&](size_t i, size_t j) {
                    return fy[i] != fy[j] ? fy[i] < fy[j] : fx[i] < fx[j];
                });
            Set S;
            for (size_t i : idx) {
                S.x.push_back(fx[i]);
                S.y.push_back(fy[i]);
                if (pup) S.pup.push_back((*pup)[i]);
                if (ap) S.ap.push_back((*ap)[i]);
            }
            return S;
        };
        const Set Us = frame(d.U_x, d.U_y, &d.U_pup, &d.U_ap);
        const Set Ps = frame(d.P_x, d.P_y, &d.P_pup, &d.P_ap);
        const Set Qs = frame(d.Q_x, d.Q_y, nullptr, nullptr);
        e.bx = d.solve_mx / 16;
        e.by = d.solve_my / 16;
        e.u_off = (int)ux.size();
        e.p_off = (int)px.size();
        e.q_off = (int)qx.size();
        ux.insert(ux.end(), Us.x.begin(), Us.x.end());
        uy.insert(uy.end(), Us.y.begin(), Us.y.end());
        up.insert(up.end(), Us.pup.begin(), Us.pup.end());
        ua.insert(ua.end(), Us.ap.begin(), Us.ap.end());
        px.insert(px.end(), Ps.x.begin(), Ps.x.end());
        py.insert(py.end(), Ps.y.begin(), Ps.y.end());
        pp.insert(pp.end(), Ps.pup.begin(), Ps.pup.end());
        pa.insert(pa.end(), Ps.ap.begin(), Ps.ap.end());
        qx.insert(qx.end(), Qs.x.begin(), Qs.x.end());
        qy.insert(qy.end(), Qs.y.begin(), Qs.y.end());
        auto band = [](const std::vector<int>& ys, int& y0, int& y1) {
            y0 = *std::min_element(ys.begin(), ys.end());
            y1 = *std::max_element(ys.begin(), ys.end());
        };
        band(Us.y, e.uy0, e.uy1);
        band(Qs.y, e.qy0, e.qy1);
        if (Ps.y.empty()) {
            e.py0 = 0;
            e.py1 = -1;
        } else {
            band(Ps.y, e.py0, e.py1);
        }
        auto push_rp = [&](const std::vector<int>& ys, int y0, int y1) {
            const int off = (int)rp.size();
            auto v = rowptr_of(ys, y0, y1);
            rp.insert(rp.end(), v.begin(), v.end());
            return off;
        };
        e.urp = push_rp(Us.y, e.uy0, e.uy1);
        e.qrp = push_rp(Qs.y, e.qy0, e.qy1);
        e.prp = push_rp(Ps.y, e.py0, e.py1);
        maxN = std::max(maxN, e.N);
        maxM = std::max(maxM, e.M);
        band_u = std::max(band_u, e.uy1 - e.uy0 + 1);
        band_p = std::max(band_p, e.py1 - e.py0 + 1);
        band_q = std::max(band_q, e.qy1 - e.qy0 + 1);
        e.qmask_off = (int)qmask.size();
        if (mr > 0) {   // Q membership per band row on the image's row grid, as 16-bit lane masks
            // x index xi = t + Bm k1 sits in lane(-slot) t, bit k1; 8 words per row, 16 on
            // the wide kernel's grids (Bm up to 20: lane-slots t + 16 s)
            const int Bm = e.bx, mx = 16 * e.bx, words = mr == 512 ? 16 : 8;
            qmask.resize(qmask.size() + (size_t)(e.qy1 - e.qy0 + 1) * words, 0u);
            for (size_t q = 0; q < Qs.x.size(); ++q) {
                const int xi = ((Qs.x[q] % mx) + mx) % mx;
                const int t = xi % Bm, k1 = xi / Bm;
                qmask[e.qmask_off + (size_t)(Qs.y[q] - e.qy0) * words + (t >> 1)] |= 1u << (16 * (t & 1) + k1);
            }
        }
        dfs.push_back(e);
    }
    D.n_used = (int)dfs.size();
    D.qmask_words = mr == 512 ? 16 : 8;
    // the wide kernel's scratch is sized for its longest grids (320 x 320), so that a
    // grid forced with apic_plan_set_df_grid always fits the workspace made with the plan
    D.max_mx = mr == 512 ? 320 : max_mx;
    D.max_mxy = mr == 512 ? 320 * 320 : max_mxy;
    D.max_N = maxN;
    D.max_M = maxM;
    D.mr = mr;
    D.band_u = band_u;
    D.band_p = band_p;
    D.band_q = band_q;
    if (qmask.empty()) qmask.push_back(0u);
    const size_t o_df = A.add(dfs);
    const size_t o_ux = A.add(ux), o_uy = A.add(uy), o_up = A.add(up), o_ua = A.add(ua);
    const size_t o_px = A.add(px), o_py = A.add(py), o_pp = A.add(pp), o_pa = A.add(pa);
    const size_t o_qx = A.add(qx), o_qy = A.add(qy), o_rp = A.add(rp);
    const size_t o_twn = A.add(twiddles(H.h)), o_twm = A.add(twiddles(H.m)), o_twN = A.add(twiddles(H.H));
    const size_t o_twr = A.add(twiddles(std::max(mr, 16)));
    const size_t o_ty6 = A.add(twiddles(96)), o_ty8 = A.add(twiddles(128)), o_ty9 = A.add(twiddles(144));
    const size_t o_ty10 = A.add(twiddles(160));
    const size_t o_w12 = A.add(twiddles(192)), o_w16 = A.add(twiddles(256)), o_w18 = A.add(twiddles(288));
    const size_t o_w20 = A.add(twiddles(320));
    const size_t o_qm = A.add(qmask);

    void* base = nullptr;
    apic_status s = dmalloc(plan, &base, A.host.size());
    if (s != APIC_OK) return s;
    APIC_TRY_CUDA(cudaMemcpy(base, A.host.data(), A.host.size(), cudaMemcpyHostToDevice));
    plan->d_tables = base;
    char* b = (char*)base;
    D.pup_x = (const int*)(b + o_pupx);
    D.pup_y = (const int*)(b + o_pupy);
    D.pup_lut = (const int*)(b + o_lut);
    D.pup_rowptr = (const int*)(b + o_puprp);
    D.led_x = (const int*)(b + o_ledx);
    D.led_y = (const int*)(b + o_ledy);
    D.led_pup = (const int*)(b + o_ledp);
    D.row_il = (const int*)(b + o_il);
    D.row_pi = (const int*)(b + o_pi);
    D.row_pl = (const int*)(b + o_pl);
    D.row_nx = (const int*)(b + o_nx);
    D.row_ny = (const int*)(b + o_ny);
    D.row_A = (const float*)(b + o_A);
    D.Lval = (const double*)(b + o_Lv);
    D.Lgrad = (const double*)(b + o_Lg);
    D.ap_x = (const int*)(b + o_apx);
    D.ap_y = (const int*)(b + o_apy);
    D.ap_bf = (const uint8_t*)(b + o_apbf);
    D.st_ptr = (const int*)(b + o_stp);
    D.st_img = (const int*)(b + o_sti);
    D.st_pup = (const int*)(b + o_stq);
    D.ap_rowptr = (const int*)(b + o_aprp);
    D.ap_colptr = (const int*)(b + o_apcp);
    D.ap_cole = (const int*)(b + o_apce);
    D.df = (const DevDF*)(b + o_df);
    D.dU_x = (const int*)(b + o_ux);
    D.dU_y = (const int*)(b + o_uy);
    D.dU_pup = (const int*)(b + o_up);
    D.dU_ap = (const int*)(b + o_ua);
    D.dP_x = (const int*)(b + o_px);
    D.dP_y = (const int*)(b + o_py);
    D.dP_pup = (const int*)(b + o_pp);
    D.dP_ap = (const int*)(b + o_pa);
    D.dQ_x = (const int*)(b + o_qx);
    D.dQ_y = (const int*)(b + o_qy);
    D.d_rowptr = (const int*)(b + o_rp);
    D.tw_n = (const float2*)(b + o_twn);
    D.tw_m = (const float2*)(b + o_twm);
    D.tw_N = (const float2*)(b + o_twN);
    D.tw_r = (const float2*)(b + o_twr);
    D.tw_y6 = (const float2*)(b + o_ty6);
    D.tw_y8 = (const float2*)(b + o_ty8);
    D.tw_y9 = (const float2*)(b + o_ty9);
    D.tw_y10 = (const float2*)(b + o_ty10);
    D.tw_w12 = (const float2*)(b + o_w12);
    D.tw_w16 = (const float2*)(b + o_w16);
    D.tw_w18 = (const float2*)(b + o_w18);
    D.tw_w20 = (const float2*)(b + o_w20);
    D.d_qmask = (const unsigned*)(b + o_qm);
    return APIC_OK;
}

apic_status configure(apic_plan* plan) {
    const DevPlan& D = plan->dev;
    Launch& L = plan->L;
    L.smem_kk = chunk_smem_bytes(D.h, D.h);
    const int bufN = std::max(2 * (kChunk / D.h) * (D.h + 1), 2 * (kChunk / D.m) * (D.m + 1));
    L.smem_df = (size_t)bufN * sizeof(float2) + (size_t)(D.h + D.m) * sizeof(float2) + 64 * sizeof(double);
    L.smem_syn = chunk_smem_bytes(D.H, D.H);
    L.smem_sim = chunk_smem_bytes(D.h, D.h);
    const int o_kk = configure_kernel(0, L.smem_kk), o_ab = configure_kernel(1, 0);
    const int o_df = configure_kernel(2, L.smem_df), o_syn = configure_kernel(3, L.smem_syn);
    const int o_sim = configure_kernel(4, L.smem_sim), o_obj = configure_kernel(5, L.smem_syn);
    if (!o_kk || !o_ab || !o_df || !o_syn || !o_sim || !o_obj) {
        cudaGetLastError();
        return fail(APIC_ECUDA, "kernel configuration (shared memory / occupancy) failed");
    }
    const int sms = plan->sms;
    // register-FFT kernels where the sizes allow them (the default), the
    // shared-memory Stockham kernels otherwise or when asked for
    plan->kkr_ok = plan->dfr_ok = false;
    if (D.h == D.w && (D.h == 64 || D.h == 128 || D.h == 256 || D.h == 512)) {
        const size_t smem = kkr_smem_bytes(D.h / 16);
        const int occ = configure_kkr(D.h / 16, smem);
        if (occ > 0) {
            plan->kkr_ok = true;
            plan->smem_kkr = smem;
            plan->grid_kkr = sms * occ;
        } else {
            cudaGetLastError();
        }
    }
    if (D.mr > 0) {
        const bool wide = D.mr == 512;
        const size_t smem = wide ? dfw_smem_bytes(D.max_N, std::max({D.band_q, D.band_p, D.band_u}))
                                 : dfr_smem_bytes(D.mr / 16, D.h / 16, D.band_u, D.band_q, D.max_N);
        int dev_max = 0;
        cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device);
        if (smem <= (size_t)dev_max && wide) {
            // blocks per tile: 1 by default (measured fastest: with 2 or 4 blocks per tile
            // fewer tiles are in flight, but the cluster barriers and the passes' rows and
            // columns split over more half-warps cost more than L2 residency gains); the
            // autotuner times 1, 2 and 4
            for (int i = 0; i < 3; ++i) {
                plan->dfw_slots[i] = configure_dfw(smem, 1 << i);
                cudaGetLastError();
            }
            const int pick = plan->dfw_slots[0] > 0 ? 0 : 1;
            if (plan->dfw_slots[pick] > 0) {
                plan->dfr_ok = true;
                plan->smem_dfr = smem;
                plan->df_cluster = 1 << pick;
                plan->grid_dfr = plan->dfw_slots[pick];
            }
        } else if (smem <= (size_t)dev_max) {
            const int occ = configure_dfr(D.mr / 16, D.h / 16, smem);
            if (occ > 0) {
                plan->dfr_ok = true;
                plan->smem_dfr = smem;
                plan->grid_dfr = sms * occ;
            } else {
                cudaGetLastError();
            }
        }
    }
    const bool legacy = (plan->params.flags & APIC_LEGACY_KERNELS) != 0;
    plan->use_kkr = plan->kkr_ok && !legacy;
    plan->use_reg = plan->dfr_ok && !legacy;
    L.grid_kk = sms * o_kk;
    L.grid_ab = sms * std::min(o_ab, 2);
    L.grid_df = sms * std::min(o_df, 2);
    L.grid_syn = sms * std::min(o_syn, o_obj);
    L.grid_sim = sms * o_sim;
    // register-transform synthesis for output sides 512 and 1024 (the Stockham kernel otherwise)
    L.grid_synr = 0;
    L.smem_synr = synr_smem_bytes(D.H);
    if (!legacy && (D.H == 512 || D.H == 1024)) {
        const int o_sr = configure_synr(D.H, L.smem_synr);
        if (o_sr > 0)
            L.grid_synr = sms * o_sr;
        else
            cudaGetLastError();
    }
    return APIC_OK;
}

apic_status alloc_workspace(apic_plan* p) {
    const DevPlan& D = p->dev;
    const size_t T = (size_t)p->max_tiles;
    apic_status s;
    if ((s = dmalloc(p, (void**)&p->xdisc, T * D.n_bf * D.npup * sizeof(float2))) != APIC_OK) return s;
    if ((s = dmalloc(p, (void**)&p->zern, T * APIC_N_ZERNIKE * sizeof(float))) != APIC_OK) return s;
    if ((s = dmalloc(p, (void**)&p->phi, T * D.npup * sizeof(float))) != APIC_OK) return s;
    if ((s = dmalloc(p, (void**)&p->spec, T * D.nap * sizeof(float2))) != APIC_OK) return s;
    if ((s = dmalloc(p, (void**)&p->status, T * sizeof(int32_t))) != APIC_OK) return s;
    if ((s = dmalloc(p, (void**)&p->c2, T * sizeof(float))) != APIC_OK) return s;
    if ((s = dmalloc(p, (void**)&p->d_counters, kCounters * sizeof(unsigned long long))) != APIC_OK) return s;
    APIC_TRY_CUDA(cudaMemset(p->d_counters, 0, kCounters * sizeof(unsigned long long)));
    if ((s = dmalloc(p, (void**)&p->d_work, 2 * sizeof(int))) != APIC_OK) return s;
    const size_t kk_blocks = (size_t)std::max(p->L.grid_kk, p->grid_kkr);
    if ((s = dmalloc(p, (void**)&p->kk_scratch, kk_blocks * D.h * D.h * sizeof(float2))) != APIC_OK) return s;
    if ((s = dmalloc(p, (void**)&p->beta_scratch, (size_t)p->L.grid_ab * D.nrows * sizeof(float))) != APIC_OK)
        return s;
    // darkfield scratch for two waves of blocks: a batch's last partial wave runs
    // beside the full waves (reconstruct) on blocks of its own
    if (p->use_reg) {
        // the wide kernel's scratch covers the most tile slots of any cluster size
        p->df_slots_alloc = D.mr == 512 ? std::max({p->dfw_slots[0], p->dfw_slots[1], p->dfw_slots[2]}) : p->grid_dfr;
        p->df_per_block = D.mr == 512 ? dfw_scratch_bytes(D) : dfr_scratch_bytes(D);
        if ((s = dmalloc(p, &p->df_scratch, 2 * (size_t)p->df_slots_alloc * p->df_per_block)) != APIC_OK) return s;
    } else {
        p->df_slots_alloc = p->L.grid_df;
        p->df_per_block = df_scratch_bytes(D);
        if ((s = dmalloc(p, &p->df_scratch, 2 * (size_t)p->L.grid_df * p->df_per_block)) != APIC_OK) return s;
    }
    int least = 0, greatest = 0;
    APIC_TRY_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    APIC_TRY_CUDA(cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, greatest));
    APIC_TRY_CUDA(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    APIC_TRY_CUDA(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    APIC_TRY_CUDA(cudaEventCreateWithFlags(&p->ev_tail, cudaEventDisableTiming));
    APIC_TRY_CUDA(cudaEventCreateWithFlags(&p->ev_pre, cudaEventDisableTiming));
    APIC_TRY_CUDA(cudaEventCreateWithFlags(&p->ev_mbe, cudaEventDisableTiming));
    APIC_TRY_CUDA(cudaStreamCreateWithPriority(&p->prep, cudaStreamNonBlocking, greatest));
    for (auto& e : p->ev_prep) APIC_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return APIC_OK;
}

// Kramers-Kronig stage on `blocks` blocks (<= 0: the plan's grid) with the given scratch.
cudaError_t launch_kk_any(apic_plan* p, int blocks, int n_tiles, const float* I, float2* xdisc, float2* scratch,
                          const int32_t* status, cudaStream_t st) {
    if (p->use_kkr)
        return launch_kk_reg(p->dev, blocks > 0 ? std::min(blocks, p->grid_kkr) : p->grid_kkr, p->smem_kkr, n_tiles,
                             I, xdisc, scratch, status, st);
    return launch_kk_grid(p->dev, blocks > 0 ? std::min(blocks, p->L.grid_kk) : p->L.grid_kk, p->L.smem_kk, n_tiles,
                          I, xdisc, scratch, status, st);
}

// Darkfield blocks of one full wave (the grid of the selected kernel).
int df_wave(const apic_plan* p) { return std::max(1, p->use_reg ? p->grid_dfr : p->L.grid_df); }

// SMs that `slots` darkfield tile slots occupy (the wide kernel: df_cluster blocks each)
int df_sms(const apic_plan* p, int slots) { return slots * (p->use_reg && p->dev.mr == 512 ? p->df_cluster : 1); }

// Darkfield stage on the tiles whose phase table starts at phi, on `grid` blocks
// (<= 0: a full wave); `second` selects the second wave of scratch blocks (for a
// launch that runs beside another one).
cudaError_t launch_df_on(apic_plan* p, int n_tiles, const float* I, const float* phi, float2* spec, int32_t* status,
                         bool second, cudaStream_t st, int grid = 0) {
    char* scratch = (char*)p->df_scratch + (second ? (size_t)p->df_slots_alloc * p->df_per_block : 0);
    const int g = grid > 0 ? std::min(grid, df_wave(p)) : df_wave(p);
    if (p->use_reg && p->dev.mr == 512)
        return launch_darkfield_wide(p->dev, p->df_cluster, g, p->smem_dfr, n_tiles, I, phi, spec, scratch,
                                     p->df_per_block, p->df_iters, p->df_tol, status, p->d_counters,
                                     p->d_work + (second ? 1 : 0), st);
    if (p->use_reg)
        return launch_darkfield_reg(p->dev, g, p->smem_dfr, n_tiles, I, phi, spec, scratch, p->df_per_block,
                                    p->df_iters, p->df_tol, status, p->d_counters, p->d_work + (second ? 1 : 0), st);
    Launch L = p->L;
    L.grid_df = g;
    return launch_darkfield(p->dev, L, n_tiles, I, phi, spec, scratch, p->df_per_block, p->df_iters, p->df_tol,
                            status, p->d_counters, st);
}

cudaError_t launch_df(apic_plan* p, int n_tiles, const float* I, float2* spec, int32_t* status, cudaStream_t st) {
    return launch_df_on(p, n_tiles, I, p->phi, spec, status, false, st);
}

apic_status check_plan(const apic_plan* plan, int n_tiles) {
    if (!plan) return fail(APIC_EINVAL, "plan is NULL");
    if (plan->host_only) return fail(APIC_EINVAL, "plan was created with APIC_HOST_ONLY");
    if (n_tiles < 0) return fail(APIC_EINVAL, "n_tiles < 0");
    return APIC_OK;
}

apic_status check_stage(const apic_plan* plan, int n_tiles) {
    apic_status s = check_plan(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (n_tiles > plan->max_tiles) return fail(APIC_EINVAL, "n_tiles exceeds the plan's max_tiles");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
        return fail(APIC_EINVAL, "current device differs from the plan's device");
    return APIC_OK;
}

#define APIC_TRY_LAUNCH(expr)                                  \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return cuda_fail(_e, #expr);    \
        ++plan->launches;                                      \
    } while (0)

// Records the start (end = 0) or stop (end = 1) event of a stage in the
// current ring slot; a no-op unless timing is on for this call.
struct StageTimer {
    apic_plan* p;
    cudaStream_t st;
    int slot = -1;
    StageTimer(apic_plan* plan, cudaStream_t s) : p(plan), st(s) {
        if (!p->timing) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
        slot = p->t_next;
        p->t_next = (p->t_next + 1) % apic_plan::kTimingSlots;
        p->t_used = std::min(p->t_used + 1, apic_plan::kTimingSlots);
    }
    void mark(int stage, int end, cudaStream_t on = nullptr) {     // on: another stream of the call
        if (slot < 0) return;
        cudaEventRecord(p->events[((size_t)slot * apic_plan::kStages + stage) * 2 + end], on ? on : st);
    }
};

// Learned-path buffers (features and network coefficients for max_tiles tiles),
// allocated on the first learned call.
apic_status learned_buffers(apic_plan* p) {
    if (p->feat) return APIC_OK;
    if (!p->kkr_ok) return fail(APIC_EINVAL, "network features need tiles of 64, 128, 256 or 512 pixels");
    if (p->dev.n_bf != 8) return fail(APIC_EINVAL, "the network takes exactly 8 NA-matching images");
    apic_status s;
    if ((s = dmalloc(p, (void**)&p->feat, (size_t)p->max_tiles * feature_floats() * sizeof(float))) != APIC_OK)
        return s;
    if ((s = dmalloc(p, (void**)&p->c_net, (size_t)p->max_tiles * APIC_N_ZERNIKE * sizeof(float))) != APIC_OK)
        return s;
    return APIC_OK;
}

// Where the host pipeline joins the order of one chunk (reconstruct): wait_main
// is waited on before the first stage of the full waves' tiles. Plain order:
// early_done is recorded once all fields are synthesized. Split order:
// field_ready[k] (when set) is recorded once the fields of MA's round k, tiles
// [k wa, (k + 1) wa) with wa = W - r, are synthesized, together with those of T
// = [m0, nt) after round 0; ml_ready (when set; then on the second stream) once
// those of ML = [ma, ml) are; the fields [ml, m0) are synthesized last. Without
// ml_ready ML is synthesized after MA's last round. With parts > 0 (split order
// only) the full waves' tiles arrive in parts of whole darkfield rounds: part g
// holds rounds [part_rounds[g - 1], part_rounds[g]) of both groups (MA's tiles
// [k wa, (k + 1) wa) and MB's [ma + k r, ma + (k + 1) r) for each round k), ready
// at part_ready[g]; each part's earlier stages run on a stream of their own as
// soon as it is in, and each round starts once its part's earlier stages end.
struct SplitHooks {
    static constexpr int kMaxParts = 16;   // = the host pipeline's part events
    static constexpr int kMaxRounds = 32;  // = the host pipeline's round events
    cudaEvent_t wait_main = nullptr;
    cudaEvent_t early_done = nullptr;
    int parts = 0;
    int part_rounds[kMaxParts] = {};
    cudaEvent_t part_ready[kMaxParts] = {};
    cudaEvent_t field_ready[kMaxRounds] = {};
    cudaEvent_t ml_ready = nullptr;
};

// Partial-wave geometry of a chunk of nt tiles: r trailing tiles (0: no split),
// m0 = nt - r, ma, the full waves' tiles that go to the W - r blocks, and ml, the
// first tile of the r blocks' last round (= ma when they take a single round).
// Only a partial wave of at most W / 2 tiles is split off: the full waves' earlier
// stages run beside its solves on the W - r SMs it leaves, which for a larger one
// would be too few (a partial wave of r > W / 2 idles fewer than W / 2 SMs for one
// round at the end of the plain order).
void split_geometry(const apic_plan* p, int nt, int& r, int& m0, int& ma, int& ml) {
    const int W = df_wave(p);
    r = (p->dev.n_used > 0 && nt > W) ? nt % W : 0;
    if (2 * r > W) r = 0;
    m0 = nt - r;
    ma = r > 0 ? (W - r) * (m0 / W) : m0;
    ml = r > 0 && m0 - ma > r ? m0 - r : ma;
}

// Background, Kramers-Kronig, aberration (learned when `net`), stitching,
// darkfield, synthesis and pupil over chunks of max_tiles tiles.
//
// The darkfield stage runs one tile per block, so a chunk of nt tiles takes
// ceil(nt / W) block rounds (W = blocks of a full wave) and its last partial
// round leaves SMs idle. When nt is not a multiple of W, the r = nt mod W
// trailing tiles go first: their earlier stages run, their darkfield solves
// start on a high-priority second stream (own scratch blocks), and meanwhile
// the earlier stages of the other tiles run on the remaining SMs. Those tiles
// then go to W - r blocks on the caller's stream (they start right away) and r
// blocks on the second stream (they start where the partial wave ends), one
// launch per round of one tile per block, so that each block takes the same
// number of tiles; every round's fields but those of the second group's last
// round are synthesized while later rounds run. Every tile gets exactly the
// computation of the plain order.
apic_status reconstruct(apic_plan* plan, apic_net* net, int mode, int n_tiles, const float* I, const float* uv,
                        float* field, float* zern, float* pupil, int32_t* status, cudaStream_t st,
                        const SplitHooks* hk = nullptr) {
    const DevPlan& D = plan->dev;
    const Launch& L = plan->L;
    const size_t in_tile = (size_t)D.n_img * D.h * D.w, out_tile = (size_t)D.H * D.W;
    const bool replace = net && (mode & APIC_NET_REPLACE);
    const bool warm = net && (mode & APIC_NET_WARM);
    const float thresh2 = replace ? plan->bg_c2 : plan->bg_thresh2;
    const int W = df_wave(plan);
    StageTimer tm(plan, st);
    for (int t0 = 0; t0 < n_tiles; t0 += plan->max_tiles) {
        const int nt = std::min(plan->max_tiles, n_tiles - t0);
        const bool first = t0 == 0, last = t0 + nt >= n_tiles;
        const float* It = I + (size_t)t0 * in_tile;
        int32_t* stt = status ? status + t0 : plan->status;
        float* zt = zern + (size_t)t0 * APIC_N_ZERNIKE;
        int r = 0, m0 = nt, ma = nt, ml = nt;   // partial wave, full waves, their groups
        split_geometry(plan, nt, r, m0, ma, ml);
        // earlier stages of tiles [a, a + k) of the chunk; in the split order this runs
        // for the partial wave (a = m0) and then for the full waves (a = 0), so a stage's
        // interval starts with the first call and ends with the call for a = 0. cap > 0
        // limits the persistent kernels (KK, aberration) to cap SMs' worth of blocks: the
        // full waves' earlier stages then never hold an SM the partial wave's darkfield
        // blocks are about to take (a persistent block keeps its SM for milliseconds)
        bool pre_first = true;
        cudaStream_t ps = st;       // stream of the earlier stages (the caller's, or the parts' own)
        auto pre_df = [&](int a, int k, bool final, int cap) -> apic_status {
            if (k == 0) return APIC_OK;
            const bool mark0 = first && pre_first, mark1 = last && final;
            pre_first = false;
            float2* xd = plan->xdisc + (size_t)a * D.n_bf * D.npup;
            float* ph = plan->phi + (size_t)a * D.npup;
            Launch La = L;
            if (cap > 0) La.grid_ab = std::min(L.grid_ab, 2 * cap);
            if (mark0) tm.mark(1, 0);
            APIC_TRY_LAUNCH(launch_kk_any(plan, cap, k, It + (size_t)a * in_tile, xd, plan->kk_scratch, stt + a, ps));
            if (mark1) tm.mark(1, 1, ps);
            if (mark0) tm.mark(2, 0);
            APIC_TRY_LAUNCH(launch_aberration(D, La, k, xd, zt + (size_t)a * APIC_N_ZERNIKE, plan->beta_scratch,
                                              plan->ab_passes, stt + a, ps,
                                              net ? plan->c_net + (size_t)a * APIC_N_ZERNIKE : nullptr, warm ? 1 : 0));
            if (mark1) tm.mark(2, 1, ps);
            if (mark0) tm.mark(3, 0);
            APIC_TRY_LAUNCH(launch_phase(D, k, zt + (size_t)a * APIC_N_ZERNIKE, ph, ps));
            APIC_TRY_LAUNCH(launch_stitch(D, k, xd, ph, plan->spec + (size_t)a * D.nap, stt + a, ps));
            if (mark1) tm.mark(3, 1, ps);
            return APIC_OK;
        };
        // network coefficients of tiles [a, a + k) of the chunk (learned path)
        auto learned_part = [&](int a, int k, int cap) -> apic_status {
            if (!net || k == 0) return APIC_OK;
            float* feat = plan->feat + (size_t)a * feature_floats();
            const int fgrid = cap > 0 ? std::min(cap, plan->grid_kkr) : plan->grid_kkr;
            APIC_TRY_LAUNCH(launch_features(D, fgrid, k, It + (size_t)a * in_tile, feat, plan->kk_scratch, ps));
            const int nb = net_max_batch(net);
            for (int b0 = 0; b0 < k; b0 += nb) {
                const int bn = std::min(nb, k - b0);
                const long long before = net_launches(net);
                APIC_TRY_CUDA(net_predict(net, bn, feat + (size_t)b0 * feature_floats(),
                                          uv + (size_t)(t0 + a + b0) * 2,
                                          plan->c_net + (size_t)(a + b0) * APIC_N_ZERNIKE, ps));
                plan->launches += net_launches(net) - before;
            }
            return APIC_OK;
        };
        // with several chunks a stage's interval spans from its first start to its last stop;
        // in the split order the intervals of the stages overlap
        apic_status s;
        float2* fld = (float2*)field + (size_t)t0 * out_tile;
        if (r > 0) {
            // Tiles of the full waves split into MA = [0, ma) on W - r blocks and
            // MB = [ma, m0) on r blocks (one tile per block per round, m0 / W rounds each); T = [m0, nt) is the
            // partial wave. Caller's stream: T's earlier stages, then (fork) the full
            // waves' background and earlier stages (with input parts: per part on a
            // stream of their own, each round waiting for its part), MA's darkfield
            // rounds, each followed by its synthesis (T's after the first, ML = [ma, ml)
            // after the last). Second stream: T's darkfield, then MB's darkfield rounds
            // and the synthesis of its last round (join).
            if (first) tm.mark(0, 0);
            APIC_TRY_LAUNCH(launch_background(D, r, It + (size_t)m0 * in_tile, plan->c2 + m0, stt + m0, thresh2, st,
                                              replace ? 1 : 0));
            if ((s = learned_part(m0, r, 0)) != APIC_OK) return s;
            if ((s = pre_df(m0, r, false, 0)) != APIC_OK) return s;
            APIC_TRY_CUDA(cudaEventRecord(plan->ev_fork, st));
            if (first) tm.mark(4, 0);
            APIC_TRY_CUDA(cudaStreamWaitEvent(plan->side, plan->ev_fork, 0));
            APIC_TRY_LAUNCH(launch_df_on(plan, r, It + (size_t)m0 * in_tile, plan->phi + (size_t)m0 * D.npup,
                                         plan->spec + (size_t)m0 * D.nap, stt + m0, true, plan->side, r));
            APIC_TRY_CUDA(cudaEventRecord(plan->ev_tail, plan->side));
            const int wa = W - r, rounds = m0 / W;
            // earlier stages of tiles [a, b) on stream ps (after the full waves' inputs, or
            // a part of them, are in)
            // (cap: SMs the persistent KK / aberration kernels may hold, 0 = all)
            auto full_pre = [&](int a, int b, bool final, int cap) -> apic_status {
                APIC_TRY_LAUNCH(launch_background(D, b - a, It + (size_t)a * in_tile, plan->c2 + a, stt + a, thresh2,
                                                  ps, replace ? 1 : 0));
                if (last && final) tm.mark(0, 1, ps);
                apic_status q;
                if ((q = learned_part(a, b - a, cap)) != APIC_OK) return q;
                return pre_df(a, b - a, final, cap);
            };
            const bool rparts = hk && hk->parts > 0;
            int round_part[SplitHooks::kMaxRounds] = {};     // part of each round (round parts)
            if (rparts) {
                if (hk->parts > SplitHooks::kMaxParts || hk->part_rounds[hk->parts - 1] != rounds)
                    return fail(APIC_EINTERNAL, "input parts do not cover the darkfield rounds");
                if (rounds > SplitHooks::kMaxRounds) return fail(APIC_EINTERNAL, "too many darkfield rounds for parts");
                // the shared KK / aberration scratch: after the partial wave's earlier stages
                APIC_TRY_CUDA(cudaStreamWaitEvent(plan->prep, plan->ev_fork, 0));
                ps = plan->prep;
                for (int g = 0, k0 = 0; g < hk->parts; ++g) {
                    const int k1 = hk->part_rounds[g];
                    APIC_TRY_CUDA(cudaStreamWaitEvent(ps, hk->part_ready[g], 0));
                    // the first part runs beside the partial wave's solves, so it leaves their
                    // SMs free; later parts run between darkfield rounds, on every SM that frees
                    const bool fin = g == hk->parts - 1;
                    const int cap = g == 0 ? df_sms(plan, W - r) : 0;
                    if ((s = full_pre(k0 * wa, k1 * wa, false, cap)) != APIC_OK) return s;
                    if ((s = full_pre(ma + k0 * r, ma + k1 * r, fin, cap)) != APIC_OK) return s;
                    APIC_TRY_CUDA(cudaEventRecord(plan->ev_prep[g], ps));
                    for (int k = k0; k < k1; ++k) round_part[k] = g;
                    k0 = k1;
                }
                ps = st;
            } else {
                if (hk && hk->wait_main) APIC_TRY_CUDA(cudaStreamWaitEvent(st, hk->wait_main, 0));
                // the first quarter capped, so that the partial wave's blocks (forked just
                // before) keep their SMs; the rest on every SM, so that the SMs the partial
                // wave frees when it ends do not idle until the full waves are prepared
                const int a1 = std::max(1, m0 / 4);
                if ((s = full_pre(0, a1, false, df_sms(plan, W - r))) != APIC_OK) return s;
                if ((s = full_pre(a1, m0, true, 0)) != APIC_OK) return s;
                APIC_TRY_CUDA(cudaEventRecord(plan->ev_pre, st));
                APIC_TRY_CUDA(cudaStreamWaitEvent(plan->side, plan->ev_pre, 0));
            }
            // a round waits for its part's earlier stages (round parts), once per part
            auto round_ready = [&](cudaStream_t x, int k, int& seen) -> cudaError_t {
                if (!rparts || round_part[k] == seen) return cudaSuccess;
                seen = round_part[k];
                return cudaStreamWaitEvent(x, plan->ev_prep[seen], 0);
            };
            int seen_b = -1, seen_a = -1;
            // MB one round (r tiles, one per block) per launch: the rounds before the
            // last are synthesized on the caller's stream with MA, so that only the
            // last round's fields remain once the second stream ends
            for (int a = ma; a < m0; a += r) {
                APIC_TRY_CUDA(round_ready(plan->side, (a - ma) / r, seen_b));
                APIC_TRY_LAUNCH(launch_df_on(plan, r, It + (size_t)a * in_tile, plan->phi + (size_t)a * D.npup,
                                             plan->spec + (size_t)a * D.nap, stt + a, true, plan->side, r));
                if (a + r == ml) {
                    APIC_TRY_CUDA(cudaEventRecord(plan->ev_mbe, plan->side));
                    if (hk && hk->ml_ready) {     // ML's fields right away, for the host pipeline
                        APIC_TRY_LAUNCH(launch_synthesize(D, L, ml - ma, plan->spec + (size_t)ma * D.nap,
                                                          fld + (size_t)ma * out_tile, stt + ma, plan->side));
                        APIC_TRY_CUDA(cudaEventRecord(hk->ml_ready, plan->side));
                    }
                }
            }
            APIC_TRY_LAUNCH(launch_synthesize(D, L, m0 - ml, plan->spec + (size_t)ml * D.nap,
                                              fld + (size_t)ml * out_tile, stt + ml, plan->side));
            APIC_TRY_CUDA(cudaEventRecord(plan->ev_join, plan->side));
            // MA one round (W - r tiles, one per block) per launch, each round's fields
            // synthesized right after it (T's after the first round, [ma, ml) after the
            // last), so that a host pipeline can copy them out while the rest runs
            for (int a = 0, k = 0; a < ma; a += wa, ++k) {
                APIC_TRY_CUDA(round_ready(st, k, seen_a));
                APIC_TRY_LAUNCH(launch_df_on(plan, wa, It + (size_t)a * in_tile, plan->phi + (size_t)a * D.npup,
                                             plan->spec + (size_t)a * D.nap, stt + a, false, st, wa));
                if (first && k == 0) tm.mark(5, 0);
                APIC_TRY_LAUNCH(launch_synthesize(D, L, wa, plan->spec + (size_t)a * D.nap, fld + (size_t)a * out_tile,
                                                  stt + a, st));
                if (k == 0) {
                    APIC_TRY_CUDA(cudaStreamWaitEvent(st, plan->ev_tail, 0));
                    APIC_TRY_LAUNCH(launch_synthesize(D, L, r, plan->spec + (size_t)m0 * D.nap,
                                                      fld + (size_t)m0 * out_tile, stt + m0, st));
                }
                if (a + wa == ma && ml > ma && !(hk && hk->ml_ready)) {
                    APIC_TRY_CUDA(cudaStreamWaitEvent(st, plan->ev_mbe, 0));
                    APIC_TRY_LAUNCH(launch_synthesize(D, L, ml - ma, plan->spec + (size_t)ma * D.nap,
                                                      fld + (size_t)ma * out_tile, stt + ma, st));
                }
                if (hk && k < SplitHooks::kMaxRounds && hk->field_ready[k])
                    APIC_TRY_CUDA(cudaEventRecord(hk->field_ready[k], st));
            }
            APIC_TRY_CUDA(cudaStreamWaitEvent(st, plan->ev_join, 0));
            if (last) tm.mark(4, 1);
            if (last) tm.mark(5, 1);
        } else {
            if (hk && hk->wait_main) APIC_TRY_CUDA(cudaStreamWaitEvent(st, hk->wait_main, 0));
            if (first) tm.mark(0, 0);
            APIC_TRY_LAUNCH(launch_background(D, nt, It, plan->c2, stt, thresh2, st, replace ? 1 : 0));
            if (last) tm.mark(0, 1);
            if ((s = learned_part(0, nt, 0)) != APIC_OK) return s;
            if ((s = pre_df(0, nt, true, 0)) != APIC_OK) return s;
            if (first) tm.mark(4, 0);
            APIC_TRY_LAUNCH(launch_df(plan, nt, It, plan->spec, stt, st));
            if (last) tm.mark(4, 1);
            if (first) tm.mark(5, 0);
            APIC_TRY_LAUNCH(launch_synthesize(D, L, nt, plan->spec, fld, stt, st));
            if (hk && hk->early_done) APIC_TRY_CUDA(cudaEventRecord(hk->early_done, st));
            if (last) tm.mark(5, 1);
        }
        if (first) tm.mark(6, 0);
        if (pupil)
            APIC_TRY_LAUNCH(launch_pupil(D, nt, plan->phi, (float2*)pupil + (size_t)t0 * D.h * D.w, stt, st));
        if (last) tm.mark(6, 1);
    }
    return APIC_OK;
}

}  // namespace

namespace apic {
int record_error(int status, const char* msg) {
    g_last_error = msg ? msg : "";
    return status;
}
}  // namespace apic

extern "C" {

const char* apic_status_string(apic_status s) {
    switch (s) {
        case APIC_OK: return "APIC_OK";
        case APIC_EINVAL: return "APIC_EINVAL: invalid argument";
        case APIC_ENOMEM: return "APIC_ENOMEM: allocation failed";
        case APIC_ECUDA: return "APIC_ECUDA: CUDA error";
        case APIC_EGEOMETRY: return "APIC_EGEOMETRY: unusable illumination geometry";
        case APIC_EINTERNAL: return "APIC_EINTERNAL: internal error";
        case APIC_ENOTCONV: return "APIC_ENOTCONV: a darkfield solve stopped above its tolerance";
    }
    return "unknown apic_status";
}

const char* apic_last_error(void) { return g_last_error.c_str(); }

apic_status apic_measure_fma_rate(int precision, double* h_flops_per_s) {
    if (!h_flops_per_s) return fail(APIC_EINVAL, "NULL output");
    if (precision != 32 && precision != 64) return fail(APIC_EINVAL, "precision must be 32 or 64");
    const cudaError_t e = measure_fma_rate(precision, h_flops_per_s);
    if (e != cudaSuccess) return cuda_fail(e, "FMA rate kernel");
    return APIC_OK;
}

apic_status apic_plan_create(const apic_params* pr, apic_plan** out) {
    if (!pr || !out) return fail(APIC_EINVAL, "NULL params or out");
    *out = nullptr;
    if (!pow2(pr->tile_h) || pr->tile_h != pr->tile_w || pr->tile_h > 1024)
        return fail(APIC_EINVAL, "tile_h == tile_w must be a power of two in [16, 1024]");
    if (pr->n_bf < 2 || pr->n_bf > 255 || pr->n_df < 0 || pr->n_df > 4096)
        return fail(APIC_EINVAL, "n_bf must be in [2, 255] and n_df in [0, 4096]");
    if (!pr->h_kx || !pr->h_ky) return fail(APIC_EINVAL, "NULL illumination arrays");
    if (!(pr->na > 0 && pr->na < 1.5f) || !(pr->wavelength_um > 0) || !(pr->pixel_um > 0))
        return fail(APIC_EINVAL, "na, wavelength_um, pixel_um must be positive");
    // the output transform takes lengths 2^k and 3 * 2^k (upsampling 3: the paper's set-up size)
    const int out_n = pr->tile_h * pr->upsample;
    if (pr->upsample < 1 || pr->upsample > 8 || !(pow2(out_n) || (out_n % 3 == 0 && pow2(out_n / 3))) || out_n > 3072)
        return fail(APIC_EINVAL, "upsample must make the output side 2^k or 3 * 2^k, at most 3072");
    if (pr->max_tiles < 1) return fail(APIC_EINVAL, "max_tiles < 1");

    apic_plan* plan = new apic_plan();
    plan->params = *pr;
    plan->max_tiles = pr->max_tiles;
    plan->df_iters = pr->df_iters > 0 ? pr->df_iters : 40;
    plan->df_tol = pr->df_tol > 0 ? pr->df_tol : 3e-4f;
    plan->ab_passes = pr->ab_passes >= 0 ? pr->ab_passes : 2;
    const float bgc = pr->bg_contrast;
    plan->bg_c2 = bgc * bgc;
    plan->bg_thresh2 = (pr->flags & APIC_SKIP_BACKGROUND) ? bgc * bgc : -1.0f;

    GeomParams g;
    g.h = pr->tile_h;
    g.w = pr->tile_w;
    g.up = pr->upsample;
    g.n_bf = pr->n_bf;
    g.n_df = pr->n_df;
    g.na = (double)pr->na;
    g.wl = (double)pr->wavelength_um;
    g.dx = (double)pr->pixel_um;
    for (int i = 0; i < pr->n_bf + pr->n_df; ++i) {
        g.kx.push_back((double)pr->h_kx[i]);
        g.ky.push_back((double)pr->h_ky[i]);
    }
    std::string err = build_host_plan(g, plan->host);
    if (!err.empty()) {
        delete plan;
        return fail(APIC_EGEOMETRY, err);
    }
    if (plan->host.m > 1024 || plan->host.m > std::max(plan->host.h, 1024)) {
        delete plan;
        return fail(APIC_EGEOMETRY, "darkfield correlation grid too large");
    }
    if (!(pr->flags & APIC_HOST_ONLY)) {
        cudaError_t e = cudaGetDevice(&plan->device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&plan->sms, cudaDevAttrMultiProcessorCount, plan->device);
        if (e != cudaSuccess) {
            delete plan;
            return cuda_fail(e, "device query");
        }
    }
    if (pr->flags & APIC_HOST_ONLY) {
        plan->host_only = true;
        *out = plan;
        return APIC_OK;
    }
    apic_status s = upload(plan);
    if (s == APIC_OK) s = configure(plan);
    if (s == APIC_OK) s = alloc_workspace(plan);
    if (s == APIC_OK) {
        // load the allocation-free entry point's static array now (first look-up on a
        // device), so that none of that entry point's calls is the one that loads it
        float2* na = nullptr;
        const cudaError_t e = noalloc_scratch(plan->device, &na);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s = cuda_fail(e, "static scratch address (cudaGetSymbolAddress)");
        }
    }
    if (s != APIC_OK) {
        apic_plan_destroy(plan);
        return s;
    }
    *out = plan;
    return APIC_OK;
}

apic_status apic_plan_destroy(apic_plan* plan) {
    if (!plan) return APIC_OK;
    if (!plan->host_only) {
        cudaDeviceSynchronize();
        for (void* p : plan->allocs) cudaFree(p);
        for (auto e : plan->events) cudaEventDestroy(e);
        if (plan->side) cudaStreamDestroy(plan->side);
        if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
        if (plan->ev_join) cudaEventDestroy(plan->ev_join);
        if (plan->ev_tail) cudaEventDestroy(plan->ev_tail);
        if (plan->ev_pre) cudaEventDestroy(plan->ev_pre);
        if (plan->ev_mbe) cudaEventDestroy(plan->ev_mbe);
        for (cudaEvent_t e : plan->ev_prep)
            if (e) cudaEventDestroy(e);
        if (plan->prep) cudaStreamDestroy(plan->prep);
        auto& io = plan->io;
        for (int b = 0; b < 2; ++b) {
            if (io.in_done[b]) cudaEventDestroy(io.in_done[b]);
            if (io.comp_done[b]) cudaEventDestroy(io.comp_done[b]);
            if (io.out_done[b]) cudaEventDestroy(io.out_done[b]);
        }
        if (io.in_tail) cudaEventDestroy(io.in_tail);
        if (io.early) cudaEventDestroy(io.early);
        for (cudaEvent_t e : io.part)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : io.rdone)
            if (e) cudaEventDestroy(e);
        if (io.ml_done) cudaEventDestroy(io.ml_done);
        if (io.s_in) cudaStreamDestroy(io.s_in);
        if (io.s_comp) cudaStreamDestroy(io.s_comp);
        if (io.s_out) cudaStreamDestroy(io.s_out);
    }
    delete plan;
    return APIC_OK;
}

apic_status apic_plan_query(const apic_plan* plan, apic_plan_info* info) {
    if (!plan || !info) return fail(APIC_EINVAL, "NULL plan or info");
    const HostPlan& H = plan->host;
    info->tile_h = H.h;
    info->tile_w = H.w;
    info->out_h = H.H;
    info->out_w = H.W;
    info->n_bf = H.n_bf;
    info->n_df = H.n_df;
    info->n_pupil = (int)H.pup_x.size();
    info->n_aperture = (int)H.ap_x.size();
    info->n_rows = (int)H.row_i.size();
    info->n_df_used = (int)std::count_if(H.df.begin(), H.df.end(), [](const DarkfieldHost& d) { return d.used; });
    info->fft_m = plan->use_reg ? H.mr : H.m;
    info->pupil_rx = H.Rx;
    info->pupil_ry = H.Ry;
    info->df_wave = plan->host_only ? 0 : df_wave(plan);
    return APIC_OK;
}

apic_status apic_plan_table(const apic_plan* plan, int which, int32_t* dst, size_t count) {
    if (!plan || !dst) return fail(APIC_EINVAL, "NULL plan or destination");
    const HostPlan& H = plan->host;
    const std::vector<int>*xs = nullptr, *ys = nullptr;
    switch (which) {
        case APIC_TABLE_LEDS: xs = &H.led_x; ys = &H.led_y; break;
        case APIC_TABLE_PUPIL: xs = &H.pup_x; ys = &H.pup_y; break;
        case APIC_TABLE_APERTURE: xs = &H.ap_x; ys = &H.ap_y; break;
        default: return fail(APIC_EINVAL, "unknown table");
    }
    if (count < 2 * xs->size()) return fail(APIC_EINVAL, "destination too small");
    for (size_t i = 0; i < xs->size(); ++i) {
        dst[2 * i] = (*xs)[i];
        dst[2 * i + 1] = (*ys)[i];
    }
    return APIC_OK;
}

apic_status apic_plan_timing(apic_plan* plan, int enable) {
    if (!plan) return fail(APIC_EINVAL, "NULL plan");
    if (plan->host_only) return fail(APIC_EINVAL, "plan was created with APIC_HOST_ONLY");
    if (enable && plan->events.empty()) {
        plan->events.resize((size_t)apic_plan::kTimingSlots * apic_plan::kStages * 2);
        for (auto& e : plan->events) APIC_TRY_CUDA(cudaEventCreate(&e));
    }
    plan->timing = enable != 0;
    return APIC_OK;
}

apic_status apic_plan_stage_ms(apic_plan* plan, double* ms, int n, int32_t* calls, int reset) {
    if (!plan || (!ms && n > 0)) return fail(APIC_EINVAL, "NULL plan or output");
    if (plan->host_only) return fail(APIC_EINVAL, "plan was created with APIC_HOST_ONLY");
    APIC_TRY_CUDA(cudaDeviceSynchronize());
    double acc[apic_plan::kStages] = {0};
    const int used = plan->t_used;
    for (int k = 0; k < used && !plan->events.empty(); ++k) {
        const int slot = ((plan->t_next - 1 - k) % apic_plan::kTimingSlots + apic_plan::kTimingSlots) %
                         apic_plan::kTimingSlots;
        for (int sidx = 0; sidx < apic_plan::kStages; ++sidx) {
            float v = 0.f;
            const cudaEvent_t a = plan->events[((size_t)slot * apic_plan::kStages + sidx) * 2];
            const cudaEvent_t b = plan->events[((size_t)slot * apic_plan::kStages + sidx) * 2 + 1];
            if (cudaEventElapsedTime(&v, a, b) == cudaSuccess) acc[sidx] += v;
            else cudaGetLastError();
        }
    }
    for (int i = 0; i < n && i < apic_plan::kStages; ++i) ms[i] = acc[i];
    if (calls) *calls = used;
    if (reset) plan->t_used = 0;
    return APIC_OK;
}

apic_status apic_plan_counters(apic_plan* plan, int64_t* out, int n, int reset) {
    if (!plan || (!out && n > 0)) return fail(APIC_EINVAL, "NULL plan or output");
    unsigned long long c[kCounters] = {};
    if (!plan->host_only) {
        APIC_TRY_CUDA(cudaDeviceSynchronize());
        APIC_TRY_CUDA(cudaMemcpy(c, plan->d_counters, sizeof(c), cudaMemcpyDeviceToHost));
        if (reset) APIC_TRY_CUDA(cudaMemset(plan->d_counters, 0, sizeof(c)));
    }
    const int used = std::min(plan->dev.n_used, kCountedImages);
    for (int i = 0; i < n && i < 3 + used; ++i)
        out[i] = i == 0 ? plan->launches : i < 3 ? (int64_t)c[i] : (int64_t)c[4 + (i - 3)];
    if (reset) plan->launches = 0;
    return APIC_OK;
}

apic_status apic_plan_df_set(const apic_plan* plan, int index, int which, int32_t* dst, size_t count,
                             int32_t* meta) {
    if (!plan) return fail(APIC_EINVAL, "NULL plan");
    const HostPlan& H = plan->host;
    if (index < 0 || index >= (int)H.df.size()) return fail(APIC_EINVAL, "darkfield index out of range");
    const DarkfieldHost& d = H.df[index];
    const std::vector<int>*xs, *ys;
    switch (which) {
        case 0: xs = &d.U_x; ys = &d.U_y; break;
        case 1: xs = &d.P_x; ys = &d.P_y; break;
        case 2: xs = &d.Q_x; ys = &d.Q_y; break;
        default: return fail(APIC_EINVAL, "which must be 0 (U), 1 (P) or 2 (Q)");
    }
    if (meta) {
        meta[0] = d.led;
        meta[1] = d.used ? 1 : 0;
        meta[2] = (int32_t)d.U_x.size();
        meta[3] = (int32_t)d.P_x.size();
        meta[4] = (int32_t)d.Q_x.size();
    }
    if (!dst) return APIC_OK;
    if (count < 2 * xs->size()) return fail(APIC_EINVAL, "destination too small");
    for (size_t i = 0; i < xs->size(); ++i) {
        dst[2 * i] = (*xs)[i];
        dst[2 * i + 1] = (*ys)[i];
    }
    return APIC_OK;
}

apic_status apic_plan_df_grid(const apic_plan* plan, int index, int32_t* h_grid) {
    if (!plan || !h_grid) return fail(APIC_EINVAL, "NULL plan or grid");
    const HostPlan& H = plan->host;
    if (index < 0 || index >= (int)H.df.size()) return fail(APIC_EINVAL, "darkfield index out of range");
    const DarkfieldHost& d = H.df[index];
    h_grid[0] = d.solve_tr;
    h_grid[1] = d.solve_mx;
    h_grid[2] = d.solve_my;
    return APIC_OK;
}

apic_status apic_plan_set_df_grid(apic_plan* plan, int index, int mx, int my) {
    if (!plan) return fail(APIC_EINVAL, "NULL plan");
    HostPlan& H = plan->host;
    if (index < 0 || index >= (int)H.df.size()) return fail(APIC_EINVAL, "darkfield index out of range");
    DarkfieldHost& d = H.df[index];
    if (!d.used) return fail(APIC_EINVAL, "darkfield image " + std::to_string(index) + " is skipped");
    if (H.mr != 192 && H.mr != 512) return fail(APIC_EINVAL, "the plan's register grid is not 192 or 512 points");
    if (!(H.mr == 192 ? df_grid_supported(mx, my) : df_wide_grid_supported(mx, my)))
        return fail(APIC_EINVAL, "unsupported darkfield grid");
    int nx = 0, ny = 0;
    df_grid_needs(d, nx, ny);
    if (mx < nx || my < ny)
        return fail(APIC_EINVAL, "grid " + std::to_string(mx) + " x " + std::to_string(my) + " aliases (needs " +
                                     std::to_string(nx) + " x " + std::to_string(ny) + ")");
    if (d.solve_mx == mx && d.solve_my == my) return APIC_OK;
    const int old_mx = d.solve_mx, old_my = d.solve_my;
    d.solve_mx = mx;
    d.solve_my = my;
    if (plan->host_only) return APIC_OK;
    // new device tables (the grid enters the per-image records and the Q lane masks);
    // the old ones are freed only once the new ones are in place, and kept (with the
    // old grid) if the upload fails
    APIC_TRY_CUDA(cudaDeviceSynchronize());
    void* old_tables = plan->d_tables;
    const DevPlan old_dev = plan->dev;
    const apic_status s = upload(plan);
    if (s != APIC_OK) {
        plan->d_tables = old_tables;
        plan->dev = old_dev;
        d.solve_mx = old_mx;
        d.solve_my = old_my;
        return s;
    }
    if (old_tables) {
        cudaFree(old_tables);
        auto it = std::find(plan->allocs.begin(), plan->allocs.end(), old_tables);
        if (it != plan->allocs.end()) plan->allocs.erase(it);
    }
    return APIC_OK;
}

apic_status apic_background(apic_plan* plan, int n_tiles, const float* I, float* c2, int32_t* status,
                            void* stream) {
    apic_status s = check_stage(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!I || !status) return fail(APIC_EINVAL, "NULL intensity or status");
    if (n_tiles == 0) return APIC_OK;
    APIC_TRY_LAUNCH(launch_background(plan->dev, n_tiles, I, c2, status, plan->bg_c2, (cudaStream_t)stream));
    return APIC_OK;
}


apic_status apic_kk_spectra(apic_plan* plan, int n_tiles, const float* I, float* xdisc, void* stream) {
    apic_status s = check_stage(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!I || !xdisc) return fail(APIC_EINVAL, "NULL intensity or output");
    if (n_tiles == 0) return APIC_OK;
    APIC_TRY_LAUNCH(launch_kk_any(plan, 0, n_tiles, I, (float2*)xdisc, plan->kk_scratch, nullptr,
                                  (cudaStream_t)stream));
    return APIC_OK;
}

apic_status apic_kk_spectra_noalloc(apic_plan* plan, int n_tiles, const float* I, float* xdisc, void* stream) {
    apic_status s = check_plan(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!I || !xdisc) return fail(APIC_EINVAL, "NULL intensity or output");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
        return fail(APIC_EINVAL, "current device differs from the plan's device");
    const size_t per_block = (size_t)plan->dev.h * plan->dev.w * sizeof(float2);
    const size_t cap = noalloc_scratch_bytes();
    if (per_block > cap)
        return fail(APIC_EINVAL, "tile of " + std::to_string(plan->dev.h) + " x " + std::to_string(plan->dev.w) +
                                     " needs " + std::to_string(per_block) + " bytes of scratch; the allocation-free"
                                     " entry point holds " + std::to_string(cap));
    if (n_tiles == 0) return APIC_OK;
    float2* scratch = nullptr;
    APIC_TRY_CUDA(noalloc_scratch(dev, &scratch));
    const int blocks = (int)std::min<size_t>(cap / per_block, (size_t)std::max(plan->L.grid_kk, plan->grid_kkr));
    APIC_TRY_LAUNCH(launch_kk_any(plan, blocks, n_tiles, I, (float2*)xdisc, scratch, nullptr, (cudaStream_t)stream));
    return APIC_OK;
}

apic_status apic_aberration(apic_plan* plan, int n_tiles, const float* xdisc, float* zern, void* stream) {
    apic_status s = check_stage(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!xdisc || !zern) return fail(APIC_EINVAL, "NULL input or output");
    if (n_tiles == 0) return APIC_OK;
    APIC_TRY_LAUNCH(launch_aberration(plan->dev, plan->L, n_tiles, (const float2*)xdisc, zern, plan->beta_scratch,
                                      plan->ab_passes, nullptr, (cudaStream_t)stream));
    return APIC_OK;
}

apic_status apic_stitch(apic_plan* plan, int n_tiles, const float* xdisc, const float* zern, float* spec,
                        void* stream) {
    apic_status s = check_stage(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!xdisc || !zern || !spec) return fail(APIC_EINVAL, "NULL argument");
    if (n_tiles == 0) return APIC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    APIC_TRY_LAUNCH(launch_phase(plan->dev, n_tiles, zern, plan->phi, st));
    APIC_TRY_LAUNCH(launch_stitch(plan->dev, n_tiles, (const float2*)xdisc, plan->phi, (float2*)spec, nullptr, st));
    return APIC_OK;
}

apic_status apic_darkfield(apic_plan* plan, int n_tiles, const float* I, const float* zern, float* spec,
                           int32_t* status, void* stream) {
    apic_status s = check_stage(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!I || !zern || !spec) return fail(APIC_EINVAL, "NULL argument");
    if (n_tiles == 0) return APIC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    APIC_TRY_LAUNCH(launch_phase(plan->dev, n_tiles, zern, plan->phi, st));
    APIC_TRY_LAUNCH(launch_df(plan, n_tiles, I, (float2*)spec, status, st));
    return APIC_OK;
}

apic_status apic_synthesize(apic_plan* plan, int n_tiles, const float* spec, float* field, void* stream) {
    apic_status s = check_stage(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!spec || !field) return fail(APIC_EINVAL, "NULL argument");
    if (n_tiles == 0) return APIC_OK;
    APIC_TRY_LAUNCH(launch_synthesize(plan->dev, plan->L, n_tiles, (const float2*)spec, (float2*)field, nullptr,
                                      (cudaStream_t)stream));
    return APIC_OK;
}

apic_status apic_pupil(apic_plan* plan, int n_tiles, const float* zern, float* pupil, void* stream) {
    apic_status s = check_stage(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!zern || !pupil) return fail(APIC_EINVAL, "NULL argument");
    if (n_tiles == 0) return APIC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    APIC_TRY_LAUNCH(launch_phase(plan->dev, n_tiles, zern, plan->phi, st));
    APIC_TRY_LAUNCH(launch_pupil(plan->dev, n_tiles, plan->phi, (float2*)pupil, nullptr, st));
    return APIC_OK;
}

apic_status apic_reconstruct_batch(apic_plan* plan, int n_tiles, const float* I, float* field, float* zern,
                                   float* pupil, int32_t* status, void* stream) {
    apic_status s = check_plan(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!I || !field || !zern) return fail(APIC_EINVAL, "NULL intensity, field or zernike buffer");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
        return fail(APIC_EINVAL, "current device differs from the plan's device");
    return reconstruct(plan, nullptr, 0, n_tiles, I, nullptr, field, zern, pupil, status, (cudaStream_t)stream);
}

apic_status apic_reconstruct_learned(apic_plan* plan, apic_net* net, int mode, int n_tiles, const float* I,
                                     const float* uv, float* field, float* zern, float* pupil, int32_t* status,
                                     void* stream) {
    apic_status s = check_plan(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!net) return fail(APIC_EINVAL, "NULL network");
    if (!I || !uv || !field || !zern) return fail(APIC_EINVAL, "NULL intensity, position, field or zernike buffer");
    if (mode & ~(APIC_NET_WARM | APIC_NET_REPLACE)) return fail(APIC_EINVAL, "unknown mode bits");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
        return fail(APIC_EINVAL, "current device differs from the plan's device");
    if ((s = learned_buffers(plan)) != APIC_OK) return s;
    return reconstruct(plan, net, mode, n_tiles, I, uv, field, zern, pupil, status, (cudaStream_t)stream);
}

apic_status apic_features(apic_plan* plan, int n_tiles, const float* I, float* feat, void* stream) {
    apic_status s = check_stage(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!I || !feat) return fail(APIC_EINVAL, "NULL intensity or features");
    if (!plan->kkr_ok) return fail(APIC_EINVAL, "network features need tiles of 64, 128, 256 or 512 pixels");
    if (plan->dev.n_bf != 8) return fail(APIC_EINVAL, "the network takes exactly 8 NA-matching images");
    if (n_tiles == 0) return APIC_OK;
    APIC_TRY_LAUNCH(launch_features(plan->dev, plan->grid_kkr, n_tiles, I, feat, plan->kk_scratch,
                                    (cudaStream_t)stream));
    return APIC_OK;
}

}  // extern "C"

namespace {
// APIC_ENOTCONV if a (host) status word of the batch has APIC_TILE_NOTCONV.
apic_status host_status_word(const int32_t* h_status, int n_tiles) {
    if (!h_status) return APIC_OK;
    for (int t = 0; t < n_tiles; ++t)
        if (h_status[t] & APIC_TILE_NOTCONV)
            return fail(APIC_ENOTCONV, "tile " + std::to_string(t) + ": a darkfield solve stopped above its tolerance");
    return APIC_OK;
}
}  // namespace

extern "C" {

apic_status apic_reconstruct_host(apic_plan* plan, int n_tiles, const float* h_I, float* h_field, float* h_zern,
                                  int32_t* h_status) {
    apic_status s = check_plan(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!h_I || !h_field || !h_zern) return fail(APIC_EINVAL, "NULL intensity, field or zernike buffer");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
        return fail(APIC_EINVAL, "current device differs from the plan's device");
    if (n_tiles == 0) return APIC_OK;
    const DevPlan& D = plan->dev;
    const size_t in_tile = (size_t)D.n_img * D.h * D.w, out_tile = (size_t)D.H * D.W;
    auto& io = plan->io;
    // A call of up to io.one tiles (normally max_tiles: the whole call's inputs and
    // fields fit on the device beside the plan) takes the one-chunk order: inputs copy
    // in parts while the earlier stages of the parts already in run, and each darkfield
    // round's fields copy out once synthesized, so the copies hide behind the
    // computation. Larger calls (or when device memory is short) go in chunks that
    // follow the darkfield grid (one tile per block): the first chunk one full wave so
    // that computation starts after a short copy, the rest up to four waves, double
    // buffered.
    const int wave = df_wave(plan);
    auto buffers = [&](int b, int C) -> apic_status {      // buffer set b for C tiles, once
        if (io.cap[b] >= C) return APIC_OK;
        if (io.cap[b] > 0) return fail(APIC_EINTERNAL, "host pipeline buffers already sized");
        void* q[4] = {};
        const size_t bytes[4] = {(size_t)C * in_tile * sizeof(float), (size_t)C * out_tile * sizeof(float2),
                                 (size_t)C * APIC_N_ZERNIKE * sizeof(float), (size_t)C * sizeof(int32_t)};
        for (int i = 0; i < 4; ++i) {
            const apic_status r = dmalloc(plan, &q[i], bytes[i]);
            if (r != APIC_OK) {          // all or nothing: a later call may try again
                for (int j = 0; j < i; ++j) {
                    cudaFree(q[j]);
                    plan->allocs.erase(std::find(plan->allocs.begin(), plan->allocs.end(), q[j]));
                }
                return r;
            }
        }
        io.d_in[b] = (float*)q[0];
        io.d_field[b] = (float*)q[1];
        io.d_zern[b] = (float*)q[2];
        io.d_status[b] = (int32_t*)q[3];
        io.cap[b] = C;
        return APIC_OK;
    };
    if (!io.ready) {
        // each object is made once: a set-up that failed part way resumes where it stopped
        auto stream = [](cudaStream_t& x) {
            return x ? cudaSuccess : cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
        };
        auto event = [](cudaEvent_t& x) {
            return x ? cudaSuccess : cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
        };
        APIC_TRY_CUDA(stream(io.s_in));
        APIC_TRY_CUDA(stream(io.s_comp));
        APIC_TRY_CUDA(stream(io.s_out));
        APIC_TRY_CUDA(event(io.in_tail));
        APIC_TRY_CUDA(event(io.early));
        for (auto& e : io.part) APIC_TRY_CUDA(event(e));
        for (auto& e : io.rdone) APIC_TRY_CUDA(event(e));
        APIC_TRY_CUDA(event(io.ml_done));
        for (int b = 0; b < 2; ++b) {
            APIC_TRY_CUDA(event(io.in_done[b]));
            APIC_TRY_CUDA(event(io.comp_done[b]));
            APIC_TRY_CUDA(event(io.out_done[b]));
        }
        io.chunk = std::max(1, std::min(plan->max_tiles, 4 * wave));
        if (io.cap[0] == 0) {
            // buffer set 0 for max_tiles tiles where that leaves a quarter of the free
            // memory (and at least 1 GiB) to others, else for one chunk
            const size_t per_tile = in_tile * sizeof(float) + out_tile * sizeof(float2) +
                                    APIC_N_ZERNIKE * sizeof(float) + sizeof(int32_t);
            size_t fr = 0, tot = 0;
            APIC_TRY_CUDA(cudaMemGetInfo(&fr, &tot));
            const size_t need = (size_t)plan->max_tiles * per_tile;
            const size_t keep = std::max(fr / 4, (size_t)1 << 30);
            const int C0 = fr > keep && need <= fr - keep ? plan->max_tiles : io.chunk;
            if ((s = buffers(0, C0)) != APIC_OK) return s;
        }
        io.one = io.cap[0];
        io.ready = true;
    }
    int r = 0, m0 = n_tiles, ma = n_tiles, ml = n_tiles;
    split_geometry(plan, n_tiles, r, m0, ma, ml);
    const bool one_order = r > 0 ? m0 / wave <= SplitHooks::kMaxRounds : n_tiles <= io.chunk;
    if (n_tiles <= io.one && one_order) {
        // One chunk, copies woven into its order: the partial darkfield wave's
        // inputs go first and its stages start while the other inputs copy; each
        // darkfield round's fields copy out as soon as they are synthesized, so that
        // only the last round's remain once the computation ends. (A whole number of
        // waves beyond one chunk has no partial wave to start with, and more rounds
        // than the round events cannot be followed: chunked order.)
        float* dI = io.d_in[0];
        float* dF = io.d_field[0];
        const size_t fbytes = out_tile * sizeof(float2);
        SplitHooks hk;
        hk.early_done = io.early;
        if (r > 0) {
            APIC_TRY_CUDA(cudaMemcpyAsync(dI + (size_t)m0 * in_tile, h_I + (size_t)m0 * in_tile,
                                          (size_t)r * in_tile * sizeof(float), cudaMemcpyHostToDevice, io.s_in));
            APIC_TRY_CUDA(cudaEventRecord(io.in_tail, io.s_in));
            // the full waves' tiles in parts of whole darkfield rounds, in the order the
            // rounds run (each round: W - r tiles of the first group, r of the second), so
            // that a round starts once its part is in and prepared while later parts copy
            static_assert(sizeof(io.part) / sizeof(io.part[0]) == SplitHooks::kMaxParts, "one event per part");
            static_assert(sizeof(io.rdone) / sizeof(io.rdone[0]) == SplitHooks::kMaxRounds, "one event per round");
            static_assert(sizeof(plan->ev_prep) / sizeof(plan->ev_prep[0]) == SplitHooks::kMaxParts, "one per part");
            const int rounds = m0 / wave, wa = wave - r;
            const int parts = std::min(SplitHooks::kMaxParts, rounds);
            auto copy_in = [&](int a, int b) -> cudaError_t {
                return cudaMemcpyAsync(dI + (size_t)a * in_tile, h_I + (size_t)a * in_tile,
                                       (size_t)(b - a) * in_tile * sizeof(float), cudaMemcpyHostToDevice, io.s_in);
            };
            for (int g = 0, k0 = 0; g < parts; ++g) {
                const int k1 = (int)((long long)rounds * (g + 1) / parts);
                APIC_TRY_CUDA(copy_in(k0 * wa, k1 * wa));
                APIC_TRY_CUDA(copy_in(ma + k0 * r, ma + k1 * r));
                APIC_TRY_CUDA(cudaEventRecord(io.part[g], io.s_in));
                hk.part_rounds[g] = k1;
                hk.part_ready[g] = io.part[g];
                k0 = k1;
            }
            hk.parts = parts;
            for (int k = 0; k < std::min(m0 / wave, SplitHooks::kMaxRounds); ++k) hk.field_ready[k] = io.rdone[k];
            hk.ml_ready = io.ml_done;
        } else {
            APIC_TRY_CUDA(cudaMemcpyAsync(dI, h_I, (size_t)m0 * in_tile * sizeof(float), cudaMemcpyHostToDevice,
                                          io.s_in));
        }
        APIC_TRY_CUDA(cudaEventRecord(io.in_done[0], io.s_in));
        APIC_TRY_CUDA(cudaStreamWaitEvent(io.s_comp, r > 0 ? io.in_tail : io.in_done[0], 0));
        s = reconstruct(plan, nullptr, 0, n_tiles, dI, nullptr, dF, io.d_zern[0], nullptr, io.d_status[0], io.s_comp,
                        &hk);
        if (s != APIC_OK) return s;
        APIC_TRY_CUDA(cudaEventRecord(io.comp_done[0], io.s_comp));
        auto fields_out = [&](int a, int k) -> cudaError_t {    // fields of tiles [a, a + k) to the host
            if (k <= 0) return cudaSuccess;
            return cudaMemcpyAsync(h_field + (size_t)a * out_tile * 2, dF + (size_t)a * out_tile * 2,
                                   (size_t)k * fbytes, cudaMemcpyDeviceToHost, io.s_out);
        };
        if (r > 0) {
            // in the order the fields become ready: MA's rounds, ML (second stream) before
            // MA's last round, then the second group's last round (rounds past the
            // round events: with the rest, once the computation ends)
            const int rounds = m0 / wave, wa = wave - r, ev_rounds = std::min(rounds, SplitHooks::kMaxRounds);
            for (int k = 0; k < ev_rounds; ++k) {
                if (k == rounds - 1 && ml > ma) {
                    APIC_TRY_CUDA(cudaStreamWaitEvent(io.s_out, io.ml_done, 0));
                    APIC_TRY_CUDA(fields_out(ma, ml - ma));
                }
                APIC_TRY_CUDA(cudaStreamWaitEvent(io.s_out, io.rdone[k], 0));
                APIC_TRY_CUDA(fields_out(k * wa, wa));
                if (k == 0) APIC_TRY_CUDA(fields_out(m0, r));
            }
            APIC_TRY_CUDA(cudaStreamWaitEvent(io.s_out, io.comp_done[0], 0));
            if (ev_rounds < rounds) {
                APIC_TRY_CUDA(fields_out(ev_rounds * wa, ma - ev_rounds * wa));
                if (ml > ma) APIC_TRY_CUDA(fields_out(ma, ml - ma));
            }
            APIC_TRY_CUDA(fields_out(ml, m0 - ml));
        } else {
            APIC_TRY_CUDA(cudaStreamWaitEvent(io.s_out, io.early, 0));
            APIC_TRY_CUDA(fields_out(0, n_tiles));
            APIC_TRY_CUDA(cudaStreamWaitEvent(io.s_out, io.comp_done[0], 0));
        }
        APIC_TRY_CUDA(cudaMemcpyAsync(h_zern, io.d_zern[0], (size_t)n_tiles * APIC_N_ZERNIKE * sizeof(float),
                                      cudaMemcpyDeviceToHost, io.s_out));
        if (h_status)
            APIC_TRY_CUDA(cudaMemcpyAsync(h_status, io.d_status[0], (size_t)n_tiles * sizeof(int32_t),
                                          cudaMemcpyDeviceToHost, io.s_out));
        APIC_TRY_CUDA(cudaStreamSynchronize(io.s_out));
        APIC_TRY_CUDA(cudaStreamSynchronize(io.s_comp));
        return host_status_word(h_status, n_tiles);
    }
    if ((s = buffers(0, io.chunk)) != APIC_OK || (s = buffers(1, io.chunk)) != APIC_OK) return s;
    int k = 0;
    for (int t0 = 0, nt = 0; t0 < n_tiles; t0 += nt, ++k) {
        nt = std::min(k == 0 ? std::min(wave, io.chunk) : io.chunk, n_tiles - t0);
        const int b = k & 1;
        // copy in once buffer b's previous reconstruction has consumed its inputs
        if (k >= 2) APIC_TRY_CUDA(cudaStreamWaitEvent(io.s_in, io.comp_done[b], 0));
        APIC_TRY_CUDA(cudaMemcpyAsync(io.d_in[b], h_I + (size_t)t0 * in_tile, (size_t)nt * in_tile * sizeof(float),
                                      cudaMemcpyHostToDevice, io.s_in));
        APIC_TRY_CUDA(cudaEventRecord(io.in_done[b], io.s_in));
        // reconstruct once the inputs are in and buffer b's previous results are out
        APIC_TRY_CUDA(cudaStreamWaitEvent(io.s_comp, io.in_done[b], 0));
        if (k >= 2) APIC_TRY_CUDA(cudaStreamWaitEvent(io.s_comp, io.out_done[b], 0));
        s = apic_reconstruct_batch(plan, nt, io.d_in[b], io.d_field[b], io.d_zern[b], nullptr, io.d_status[b],
                                   io.s_comp);
        if (s != APIC_OK) return s;
        APIC_TRY_CUDA(cudaEventRecord(io.comp_done[b], io.s_comp));
        // copy out
        APIC_TRY_CUDA(cudaStreamWaitEvent(io.s_out, io.comp_done[b], 0));
        APIC_TRY_CUDA(cudaMemcpyAsync(h_field + (size_t)t0 * out_tile * 2, io.d_field[b],
                                      (size_t)nt * out_tile * sizeof(float2), cudaMemcpyDeviceToHost, io.s_out));
        APIC_TRY_CUDA(cudaMemcpyAsync(h_zern + (size_t)t0 * APIC_N_ZERNIKE, io.d_zern[b],
                                      (size_t)nt * APIC_N_ZERNIKE * sizeof(float), cudaMemcpyDeviceToHost, io.s_out));
        if (h_status)
            APIC_TRY_CUDA(cudaMemcpyAsync(h_status + t0, io.d_status[b], (size_t)nt * sizeof(int32_t),
                                          cudaMemcpyDeviceToHost, io.s_out));
        APIC_TRY_CUDA(cudaEventRecord(io.out_done[b], io.s_out));
    }
    APIC_TRY_CUDA(cudaStreamSynchronize(io.s_out));
    APIC_TRY_CUDA(cudaStreamSynchronize(io.s_comp));
    return host_status_word(h_status, n_tiles);
}

apic_status apic_plan_autotune(apic_plan* plan, int n_tiles, const float* I, double* h_ms, int n_ms) {
    apic_status s = check_stage(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!I || n_tiles < 1) return fail(APIC_EINVAL, "autotuning needs at least one sample tile");
    APIC_TRY_CUDA(cudaDeviceSynchronize());
    cudaStream_t st = nullptr;
    APIC_TRY_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // KK register / Stockham, darkfield register / Stockham, wide darkfield kernel with 1, 2, 4 blocks per tile
    double ms[7] = {-1.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0};
    const DevPlan& D = plan->dev;
    int32_t* stt = plan->status;
    auto timed = [&](auto&& launch, double& out) -> cudaError_t {
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {       // first run warms up, best of the other two
            cudaEventRecord(e0, st);
            cudaError_t e = launch();
            if (e != cudaSuccess) return e;
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) best = std::min(best, t);
        }
        out = best;
        return cudaSuccess;
    };
    cudaError_t err = launch_background(D, n_tiles, I, plan->c2, stt, plan->bg_thresh2, st);
    // Kramers-Kronig variants (the scratch covers both grids)
    for (int v = 0; v < 2 && err == cudaSuccess; ++v) {
        if (v == 0 && !plan->kkr_ok) continue;
        plan->use_kkr = v == 0;
        err = timed([&] { return launch_kk_any(plan, 0, n_tiles, I, plan->xdisc, plan->kk_scratch, stt, st); },
                    ms[v]);
    }
    if (err == cudaSuccess) plan->use_kkr = plan->kkr_ok && !(ms[1] >= 0 && ms[1] < ms[0]);
    // inputs of the darkfield stage
    if (err == cudaSuccess) err = launch_kk_any(plan, 0, n_tiles, I, plan->xdisc, plan->kk_scratch, stt, st);
    if (err == cudaSuccess)
        err = launch_aberration(D, plan->L, n_tiles, plan->xdisc, plan->zern, plan->beta_scratch, plan->ab_passes,
                                stt, st);
    if (err == cudaSuccess) err = launch_phase(D, n_tiles, plan->zern, plan->phi, st);
    if (err == cudaSuccess) err = launch_stitch(D, n_tiles, plan->xdisc, plan->phi, plan->spec, stt, st);
    // darkfield variants, each with its own scratch; the solve is idempotent on the
    // stitched spectrum, so repeated runs see the same system
    const bool had_reg = plan->use_reg;
    const bool wide = D.mr == 512;
    const int had_k = plan->df_cluster, had_grid = plan->grid_dfr;
    void* scratch[2] = {nullptr, nullptr};
    size_t per_block[2] = {wide ? dfw_scratch_bytes(D) : dfr_scratch_bytes(D), df_scratch_bytes(D)};
    const int slots_alloc[2] = {
        wide ? std::max({plan->dfw_slots[0], plan->dfw_slots[1], plan->dfw_slots[2]}) : plan->grid_dfr,
        plan->L.grid_df};
    scratch[had_reg ? 0 : 1] = plan->df_scratch;
    int best_k = had_k, best_grid = had_grid;
    for (int v = 0; v < 2 && err == cudaSuccess; ++v) {
        if (v == 0 && !plan->dfr_ok) continue;
        if (!scratch[v]) {
            const size_t bytes = 2 * (size_t)slots_alloc[v] * per_block[v];
            if ((s = dmalloc(plan, &scratch[v], bytes)) != APIC_OK) break;
        }
        plan->use_reg = v == 0;
        plan->df_scratch = scratch[v];
        plan->df_per_block = per_block[v];
        plan->df_slots_alloc = slots_alloc[v];
        if (v == 0 && wide) {      // the wide kernel at each cluster size: blocks per tile 1, 2, 4
            for (int i = 0; i < 3 && err == cudaSuccess; ++i) {
                if (plan->dfw_slots[i] <= 0) continue;
                plan->df_cluster = 1 << i;
                plan->grid_dfr = plan->dfw_slots[i];
                err = timed([&] { return launch_df(plan, n_tiles, I, plan->spec, stt, st); }, ms[4 + i]);
                if (err == cudaSuccess && (ms[2] < 0 || ms[4 + i] < ms[2])) {
                    ms[2] = ms[4 + i];
                    best_k = plan->df_cluster;
                    best_grid = plan->grid_dfr;
                }
            }
            plan->df_cluster = best_k;
            plan->grid_dfr = best_grid;
        } else {
            err = timed([&] { return launch_df(plan, n_tiles, I, plan->spec, stt, st); }, ms[2 + v]);
        }
    }
    if (s == APIC_OK && err == cudaSuccess) {
        const int pick = plan->dfr_ok && !(ms[3] >= 0 && ms[3] < ms[2]) ? 0 : 1;
        plan->use_reg = pick == 0;
        plan->df_scratch = scratch[pick];
        plan->df_per_block = per_block[pick];
        plan->df_slots_alloc = slots_alloc[pick];
        void* loser = scratch[1 - pick];
        if (loser) {
            cudaFree(loser);
            auto it = std::find(plan->allocs.begin(), plan->allocs.end(), loser);
            if (it != plan->allocs.end()) plan->allocs.erase(it);
        }
    } else {   // keep the plan's original darkfield selection
        plan->use_reg = had_reg;
        plan->df_scratch = scratch[had_reg ? 0 : 1];
        plan->df_per_block = per_block[had_reg ? 0 : 1];
        plan->df_slots_alloc = slots_alloc[had_reg ? 0 : 1];
        plan->df_cluster = had_k;
        plan->grid_dfr = had_grid;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (s != APIC_OK) return s;
    if (err != cudaSuccess) return cuda_fail(err, "apic_plan_autotune");
    for (int i = 0; i < n_ms && i < 7; ++i) h_ms[i] = ms[i];
    return APIC_OK;
}

apic_status apic_cut_tiles(apic_plan* plan, int n_tiles, const float* slide, int slide_h, int slide_w,
                           const int32_t* windows, float* I, void* stream) {
    apic_status s = check_plan(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!slide || !windows || !I) return fail(APIC_EINVAL, "NULL slide, windows or output");
    if (slide_h < plan->dev.h || slide_w < plan->dev.w) return fail(APIC_EINVAL, "slide smaller than a tile");
    if (n_tiles == 0) return APIC_OK;
    APIC_TRY_LAUNCH(launch_cut_tiles(plan->dev, n_tiles, slide, slide_h, slide_w, windows, I, (cudaStream_t)stream));
    return APIC_OK;
}

apic_status apic_paste_fields(apic_plan* plan, int n_tiles, const float* field, const int32_t* windows, int slide_h,
                              int slide_w, float* slide_field, void* stream) {
    apic_status s = check_plan(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!field || !windows || !slide_field) return fail(APIC_EINVAL, "NULL field, windows or output");
    if (slide_h < plan->dev.h || slide_w < plan->dev.w) return fail(APIC_EINVAL, "slide smaller than a tile");
    if (n_tiles == 0) return APIC_OK;
    APIC_TRY_LAUNCH(launch_paste_fields(plan->dev, n_tiles, (const float2*)field, windows, slide_h, slide_w,
                                        (float2*)slide_field, (cudaStream_t)stream));
    return APIC_OK;
}

apic_status apic_blend_fields(apic_plan* plan, int n_tiles, const float* field, const int32_t* windows, int n_rows,
                              int n_cols, int slide_h, int slide_w, float* corr, float* phase, float* slide_field,
                              void* stream) {
    apic_status s = check_plan(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!field || !windows || !corr || !phase || !slide_field)
        return fail(APIC_EINVAL, "NULL field, windows, correlation, phase or output");
    if (n_rows < 1 || n_cols < 1 || (long long)n_rows * n_cols != n_tiles)
        return fail(APIC_EINVAL, "n_tiles must be n_rows x n_cols (the slide's whole window grid)");
    if (slide_h < plan->dev.h || slide_w < plan->dev.w) return fail(APIC_EINVAL, "slide smaller than a tile");
    APIC_TRY_LAUNCH(launch_blend(plan->dev, n_tiles, n_rows, n_cols, (const float2*)field, windows, slide_h, slide_w,
                                 (float2*)corr, (float2*)phase, (float2*)slide_field, (cudaStream_t)stream));
    return APIC_OK;
}

apic_status apic_simulate(apic_plan* plan, int n_tiles, const float* obj, const float* zern, float photons,
                          uint64_t seed, float* I, void* stream) {
    apic_status s = check_plan(plan, n_tiles);
    if (s != APIC_OK) return s;
    if (!obj || !zern || !I) return fail(APIC_EINVAL, "NULL argument");
    if (!(photons >= 0)) return fail(APIC_EINVAL, "photons must be >= 0");
    const DevPlan& D = plan->dev;
    const int chunk = std::min(plan->max_tiles, 64);
    const size_t need = ((size_t)chunk * D.H * D.W + (size_t)plan->L.grid_sim * D.h * D.w) * sizeof(float2);
    if (plan->sim_bytes < need) {
        if (plan->sim_scratch) {
            APIC_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
            cudaFree(plan->sim_scratch);
            plan->allocs.erase(std::find(plan->allocs.begin(), plan->allocs.end(), (void*)plan->sim_scratch));
            plan->sim_scratch = nullptr;
            plan->sim_bytes = 0;
        }
        if ((s = dmalloc(plan, (void**)&plan->sim_scratch, need)) != APIC_OK) return s;
        plan->sim_bytes = need;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t in_tile = (size_t)D.n_img * D.h * D.w, obj_tile = (size_t)D.H * D.W;
    for (int t0 = 0; t0 < n_tiles; t0 += chunk) {
        const int nt = std::min(chunk, n_tiles - t0);
        APIC_TRY_LAUNCH(launch_phase(D, nt, zern + (size_t)t0 * APIC_N_ZERNIKE, plan->phi, st));
        APIC_TRY_LAUNCH(launch_sim(D, plan->L, nt, (const float2*)obj + (size_t)t0 * obj_tile, plan->phi, photons,
                                   (unsigned long long)seed + (unsigned long long)t0 * 0x100000001ull,
                                   I + (size_t)t0 * in_tile, plan->sim_scratch, st));
    }
    return APIC_OK;
}

}  // extern "C"
