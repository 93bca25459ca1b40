// C-ABI of libfdtd (declared in include/fdtd.h): handle life cycle, host
// set-up in FP64 (coefficients, CPML grading, incident-wave and DFT phase
// tables) and the run loop that feeds the field-update kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fdtd_internal.h"

using namespace fdtd;

namespace fdtd {

constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
const double kMu0 = 4.0e-7 * kPi;
const double kEps0 = 1.0 / (kMu0 * kC0 * kC0);
const double kEta0 = kMu0 * kC0;
constexpr int64_t kChunk = 1024;   // steps per incident-table chunk

thread_local std::string g_create_err;

#define CK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);           \
            throw Fail{e_ == cudaErrorMemoryAllocation ? FDTD_ENOMEM : FDTD_ECUDA}; \
        }                                                                          \
    } while (0)

#define REQUIRE(cond, msg)               \
    do {                                 \
        if (!(cond)) {                   \
            h->err = (msg);              \
            throw Fail{FDTD_EINVAL};     \
        }                                \
    } while (0)

#ifdef FDTD_DEBUG_BOUNDS
// Guarded allocations of debug builds: user pointer -> (allocation base,
// user bytes), process-wide, so dfree finds the base of any buffer.
std::mutex g_guard_mu;
std::map<void*, std::pair<void*, size_t>> g_guarded;
#endif

template <typename T>
void dalloc(fdtd_handle* h, T** p, size_t count) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
#ifdef FDTD_DEBUG_BOUNDS
    const size_t user = (bytes + kGuardBytes - 1) / kGuardBytes * kGuardBytes;
    unsigned char* base = nullptr;
    CK(cudaMalloc(reinterpret_cast<void**>(&base), user + 2 * kGuardBytes));
    CK(cudaMemsetAsync(base, kGuardByte, kGuardBytes, h->stream));
    CK(cudaMemsetAsync(base + kGuardBytes + bytes, kGuardByte, user - bytes + kGuardBytes,
                       h->stream));
    *p = reinterpret_cast<T*>(base + kGuardBytes);
    {
        std::lock_guard<std::mutex> lk(g_guard_mu);
        g_guarded[*p] = std::make_pair((void*)base, bytes);
    }
    h->guarded.push_back(*p);
#else
    CK(cudaMalloc(reinterpret_cast<void**>(p), bytes));
#endif
    CK(cudaMemsetAsync(*p, 0, bytes, h->stream));
}

template <typename T>
void dfree(T*& p) {
    if (!p) return;
#ifdef FDTD_DEBUG_BOUNDS
    {
        std::lock_guard<std::mutex> lk(g_guard_mu);
        auto it = g_guarded.find((void*)p);
        if (it != g_guarded.end()) {
            cudaFree(it->second.first);
            g_guarded.erase(it);
            p = nullptr;
            return;
        }
    }
#endif
    cudaFree(p);
    p = nullptr;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// CFS-CPML recursion coefficients at a depth (cells from the interface).
void cpml_coeffs(const fdtd_grid& g, double depth, float* b, float* c, float* ik) {
    const double x = depth / (double)g.pml_cells;
    const double xm = std::pow(x, g.pml_order);
    const double sig = g.pml_sigma_max * xm;
    const double kap = 1.0 + (g.pml_kappa_max - 1.0) * xm;
    const double alp = g.pml_alpha_max * (1.0 - x);
    const double bb = std::exp(-(sig / kap + alp) * g.dt / kEps0);
    const double den = sig * kap + kap * kap * alp;
    const double cc = (sig > 0.0 && den > 0.0) ? sig * (bb - 1.0) / den : 0.0;
    *b = (float)bb;
    *c = (float)cc;
    *ik = (float)(1.0 / kap);
}

StepArgs step_args(fdtd_handle* h) {
    StepArgs a{};
    a.nx = h->g.nx; a.ny = h->g.ny; a.pitch = h->pitch; a.lpitch = h->lpitch;
    a.P = h->g.pml_cells; a.js = h->g.tfsf_row; a.jr = h->g.r_row; a.jt = h->g.t_row;
    a.n_labels = h->n_labels; a.pol = h->src.polarization; a.S = (float)h->S;
    a.labels = h->labels; a.coef = h->coef; a.cellcoef = h->cellcoef;
    a.pml_e = h->pml_e; a.pml_h = h->pml_h;
    a.hinc = h->d_hinc; a.einc = h->d_einc; a.phE = h->d_phE; a.phH = h->d_phH;
    a.dft = h->dft;
    a.n_tab = table_limit(h);
    a.n_coef = h->src.polarization == FDTD_POL_P ? 256 : h->n_labels;
    a.dbg = h->d_dbg;
    return a;
}

int64_t table_limit(const fdtd_handle* h) {
    return h->dbg_tab_limit > 0 ? std::min(h->tab_cap, h->dbg_tab_limit) : h->tab_cap;
}

void debug_checks(fdtd_handle* h) {
#ifdef FDTD_DEBUG_BOUNDS
    // guard bands of every buffer of the handle: bit 31 of the error word
    for (void* u : h->guarded) {
        std::pair<void*, size_t> g;
        {
            std::lock_guard<std::mutex> lk(g_guard_mu);
            auto it = g_guarded.find(u);
            if (it == g_guarded.end()) continue;
            g = it->second;
        }
        const size_t user = (g.second + kGuardBytes - 1) / kGuardBytes * kGuardBytes;
        const unsigned char* base = static_cast<const unsigned char*>(g.first);
        launch_guard_check(base, kGuardBytes, kGuardByte, h->d_dbg, 31, h->stream);
        launch_guard_check(base + kGuardBytes + g.second, user - g.second + kGuardBytes,
                           kGuardByte, h->d_dbg, 31, h->stream);
    }
    unsigned word = 0;
    CK(cudaMemcpyAsync(&word, h->d_dbg, sizeof word, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (word) {
        static const char* names[8] = {"lane columns", "stored row", "CPML carry row",
                                       "table entry", "monitor column", "label",
                                       "adjoint tape row", "task"};
        std::string msg = "debug checks failed:";
        for (int b = 0; b < 8; ++b)
            if (word & (1u << b)) msg += std::string(" [index check: ") + names[b] + "]";
        if (word & (1u << 31)) msg += " [guard band overwritten]";
        h->err = msg;
        throw Fail{FDTD_EBOUNDS};
    }
#else
    (void)h;
#endif
}

// Grow the incident/phase tables so that steps [0, n_end) can be produced.
void ensure_tables(fdtd_handle* h, int64_t n_end) {
    if (n_end <= h->tab_plan) return;
    int64_t plan = h->tab_plan > 0 ? std::max(n_end, 2 * h->tab_plan) : n_end;
    if (plan > h->tab_cap) {
        CK(cudaStreamSynchronize(h->stream));
        CK(cudaStreamSynchronize(h->twin_stream));
        int64_t cap = std::max<int64_t>(plan, 4096);
        float *dh = nullptr, *de = nullptr, *hh = nullptr, *he = nullptr;
        double2 *dpe = nullptr, *dph = nullptr, *hpe = nullptr, *hph = nullptr;
        CK(cudaMalloc(&dh, cap * sizeof(float)));
        CK(cudaMalloc(&de, cap * sizeof(float)));
        CK(cudaMalloc(&dpe, cap * sizeof(double2)));
        CK(cudaMalloc(&dph, cap * sizeof(double2)));
        CK(cudaMallocHost(&hh, cap * sizeof(float)));
        CK(cudaMallocHost(&he, cap * sizeof(float)));
        CK(cudaMallocHost(&hpe, cap * sizeof(double2)));
        CK(cudaMallocHost(&hph, cap * sizeof(double2)));
        if (h->tab_uploaded > 0) {
            CK(cudaMemcpy(dh, h->d_hinc, h->tab_uploaded * sizeof(float), cudaMemcpyDeviceToDevice));
            CK(cudaMemcpy(de, h->d_einc, h->tab_uploaded * sizeof(float), cudaMemcpyDeviceToDevice));
            CK(cudaMemcpy(dpe, h->d_phE, h->tab_uploaded * sizeof(double2), cudaMemcpyDeviceToDevice));
            CK(cudaMemcpy(dph, h->d_phH, h->tab_uploaded * sizeof(double2), cudaMemcpyDeviceToDevice));
        }
        dfree(h->d_hinc); dfree(h->d_einc); dfree(h->d_phE); dfree(h->d_phH);
        if (h->h_hinc) cudaFreeHost(h->h_hinc);
        if (h->h_einc) cudaFreeHost(h->h_einc);
        if (h->h_phE) cudaFreeHost(h->h_phE);
        if (h->h_phH) cudaFreeHost(h->h_phH);
        h->d_hinc = dh; h->d_einc = de; h->d_phE = dpe; h->d_phH = dph;
        h->h_hinc = hh; h->h_einc = he; h->h_phE = hpe; h->h_phH = hph;
        h->tab_cap = cap;
    }
    h->tab_plan = plan;
}

// Host part: compute incident and phase table entries up to step `upto`
// into the pinned buffers (no CUDA calls; handles may run in parallel).
void compute_tables(fdtd_handle* h, int64_t upto) {
    if (h->tab_m >= upto) return;
    TableStore& st = *h->tables;
    std::lock_guard<std::mutex> lk(st.mu);
    const int64_t have = (int64_t)st.hinc.size();
    if (have < upto) {
        if (upto > st.gen.plan_end) {
            // a longer plan: restart the generator and run it up to the
            // values already stored (they stay valid), then extend them
            st.gen.reset(std::max(h->tab_plan, 2 * st.gen.plan_end));
            float hv, ev;
            while (st.gen.m < have) st.gen.step(&hv, &ev);
        }
        st.hinc.resize(upto); st.einc.resize(upto);
        st.phE.resize(upto); st.phH.resize(upto);
        while (st.gen.m < upto) {
            const int64_t m = st.gen.m;
            st.gen.step(&st.hinc[m], &st.einc[m]);
            const double aE = st.omega * ((double)m + 0.5) * st.gen.dt;
            const double aH = st.omega * ((double)m + 1.0) * st.gen.dt;
            st.phE[m] = make_double2(std::cos(aE), std::sin(aE));
            st.phH[m] = make_double2(std::cos(aH), std::sin(aH));
        }
    }
    const int64_t m0 = h->tab_m;
    std::copy(st.hinc.begin() + m0, st.hinc.begin() + upto, h->h_hinc + m0);
    std::copy(st.einc.begin() + m0, st.einc.begin() + upto, h->h_einc + m0);
    std::copy(st.phE.begin() + m0, st.phE.begin() + upto, h->h_phE + m0);
    std::copy(st.phH.begin() + m0, st.phH.begin() + upto, h->h_phH + m0);
    h->tab_m = upto;
}

std::shared_ptr<TableStore> table_store(const IncidentGen& p, double omega) {
    using Key = std::tuple<int, double, double, double, double, double>;
    static std::mutex mu;
    static std::map<Key, std::weak_ptr<TableStore>> reg;
    const Key key{p.kind, p.S, p.dt, p.lambda0, p.bw, p.t0_over_tau};
    std::lock_guard<std::mutex> lk(mu);
    for (auto it = reg.begin(); it != reg.end();) it = it->second.expired() ? reg.erase(it) : ++it;
    if (auto sp = reg[key].lock()) return sp;
    auto sp = std::make_shared<TableStore>();
    sp->gen = p;
    sp->gen.reset(0);
    sp->omega = omega;
    reg[key] = sp;
    return sp;
}

// Queue the upload of the computed entries not yet on the device.
void upload_tables(fdtd_handle* h, int64_t upto) {
    const int64_t from = h->tab_uploaded;
    if (upto > from) {
        const int64_t cnt = upto - from;
        CK(cudaMemcpyAsync(h->d_hinc + from, h->h_hinc + from, cnt * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->d_einc + from, h->h_einc + from, cnt * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->d_phE + from, h->h_phE + from, cnt * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->d_phH + from, h->h_phH + from, cnt * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
        h->tab_uploaded = upto;
    }
}

// Compute table entries up to step `upto` and queue their upload.
void produce_tables(fdtd_handle* h, int64_t upto) {
    compute_tables(h, upto);
    upload_tables(h, upto);
}

int sm_count(fdtd_handle* h) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) v = 148;
    return v;
}

// Cost of a general-path iteration of the blocked kernel in lean
// iterations, per polarisation (S, P), as used by the segment planner. The
// general path (CPML recursion, source and monitor terms, row checks) costs
// many lean iterations; a P lean iteration does more work (label-pair
// lookups of the edge coefficients), so its ratio is lower. Measured on
// GB300 on config 2 (Gcell-updates/s, 8192 steps per run): S with code
// shape 5 (the S default): 9: 1350, 10: 1462, 11: 1521, 12: 1543, 13: 1385,
// 15: 1268, and with the skewed two-row trip 11: 1539, 12: 1604, 13: 1407;
// P with code shape 5 and the skewed trip 6.5: 1152, 7.5: 1281, 8.5: 1318,
// 9: 1239. Away from the best weight the cuts shift whole general-path rows
// between tasks, so the response is uneven.
constexpr double kGeneralCost[2] = {12.0, 8.5};

double general_cost(int pol, double override_w) {
    return override_w > 0.0 ? override_w : kGeneralCost[pol ? 1 : 0];
}

// Estimated cost of one pipeline iteration t of the warp task of a segment
// starting at y0: the kernel's lean-path test (blocked_task, is_fast) gives
// 1, the general path `wg` lean iterations. A segment [y0, y1) runs the
// iterations t_begin(y0) .. y1+K-1.
double iteration_cost(const fdtd_grid& g, int K, int t, double wg) {
    const int P = g.pml_cells;
    bool f = (t >= std::max(K + 1, P + K)) && (t < g.ny - P + 1);
    const int sp[5] = {g.tfsf_row, g.r_row, g.r_row + 1, g.t_row, g.t_row + 1};
    for (int q = 0; q < 5 && f; ++q) f = (unsigned)(t - sp[q] - 1) >= (unsigned)K;
    return f ? 1.0 : wg;
}

// Segment boundaries for about ny/seg segments of equal estimated cost for
// K steps per launch and polarisation pol. Every boundary lies in [K, ny)
// (a segment's K halo rows above it exist) and none falls on r_row + 1 or
// t_row + 1 (the segment owning a monitor row also owns the row below it,
// whose Hx enters the row average).
std::vector<int> segment_bounds(const fdtd_grid& g, int seg, int K, int pol, double weight) {
    const int ny = g.ny;
    const int n_target = std::max(1, (int)std::lround((double)ny / std::max(seg, 1)));
    const double wg = general_cost(pol, weight);
    // prefix sums of the iteration costs: a segment [y0, y1) costs
    // C(y1 + K) - C(t_begin(y0))
    std::vector<double> C((size_t)ny + K + 1, 0.0);
    for (int t = 0; t < ny + K; ++t) C[(size_t)t + 1] = C[(size_t)t] + iteration_cost(g, K, t, wg);
    auto cost = [&](int y0, int y1) { return C[(size_t)y1 + K] - C[(size_t)(y0 == 0 ? 0 : y0 - K)]; };
    auto ok_cut = [&](int y) {
        return y >= K && y >= 1 && y < ny && y != g.r_row + 1 && y != g.t_row + 1;
    };
    // greedy cut with every segment cost <= T; empty when more than
    // n_target segments would be needed
    auto cut = [&](double T) {
        std::vector<int> b{0};
        int y0 = 0;
        while (cost(y0, ny) > T) {
            int best = -1;
            for (int y1 = y0 + 1; y1 < ny; ++y1) {
                if (cost(y0, y1) > T) break;
                if (ok_cut(y1)) best = y1;
            }
            if (best < 0 || (int)b.size() >= n_target) return std::vector<int>();
            b.push_back(best);
            y0 = best;
        }
        b.push_back(ny);
        return b;
    };
    double lo = 0.0, hi = cost(0, ny);
    std::vector<int> best{0, ny};
    for (int it = 0; it < 50 && hi - lo > 0.25; ++it) {
        const double mid = 0.5 * (lo + hi);
        std::vector<int> b = cut(mid);
        if (b.empty()) {
            lo = mid;
        } else {
            hi = mid;
            best = b;
        }
    }
    // Segments the layout rules keep from splitting can bound the maximum
    // cost; use the rest of the segment budget anyway, splitting the
    // costliest splittable segment where its halves cost the same (the
    // maximum does not grow, the tasks fill the GPU).
    while ((int)best.size() - 1 < n_target) {
        int pick = -1, at = -1;
        double pick_cost = -1.0;
        for (size_t q = 0; q + 1 < best.size(); ++q) {
            const int y0 = best[q], y1 = best[q + 1];
            const double c = cost(y0, y1);
            if (c <= pick_cost) continue;
            int m = -1;
            double bal = 1e300;
            for (int y = y0 + 1; y < y1; ++y) {
                if (!ok_cut(y)) continue;
                const double d = std::fabs(cost(y0, y) - cost(y, y1));
                if (d < bal) { bal = d; m = y; }
            }
            if (m < 0) continue;
            pick = (int)q;
            at = m;
            pick_cost = c;
        }
        if (pick < 0) break;
        best.insert(best.begin() + pick + 1, at);
    }
    return best;
}

// Segment plan of the blocked kernel for depth K (see blocked.cu). One warp
// task per (strip, segment); with W warps resident on the whole GPU, the
// segment count is chosen to minimise waves x (rows per segment + 2K), the
// cost model of a wave of equal tasks that each stream their rows plus
// the K-row halos above and below. `cache` holds one plan per depth for
// code shape `variant` and planner weight `weight` (0: the default of the
// polarisation).
BlockPlan& plan_for(fdtd_handle* h, std::vector<BlockPlan>& cache, int K, int variant,
                    double weight) {
    if ((int)cache.size() <= K) cache.resize(K + 1);
    BlockPlan& p = cache[K];
    const int want_seg = h->opt_seg;
    if (p.K == K && p.d_seg_y0 && p.variant == variant && p.weight == weight &&
        (want_seg == 0 || want_seg == p.seg_rows))
        return p;
    dfree(p.d_seg_y0);
    const fdtd_grid& g = h->g;
    p.K = K;
    p.variant = variant;
    p.weight = weight;
    p.halo = (K + 3) / 4 * 4;
    p.w_int = 128 - 2 * p.halo;
    p.n_strips = (g.nx + p.w_int - 1) / p.w_int;
    const int min_seg = K + 1;
    int seg = want_seg;
    if (seg <= 0) {
        int per_sm = blocked_warps_per_sm(K, variant, h->src.polarization);
        if (per_sm <= 0) per_sm = 8;
        const int64_t W = (int64_t)sm_count(h) * per_sm;
        double best = 1e300;
        seg = g.ny;
        const int max_n = std::max(1, g.ny / min_seg);
        for (int n = 1; n <= max_n; ++n) {
            const int64_t tasks = (int64_t)n * p.n_strips;
            const int64_t waves = (tasks + W - 1) / W;
            const double rows = std::ceil((double)g.ny / n);
            const double cost = (double)waves * (rows + 2.0 * K);
            if (cost < best - 1e-9) {
                best = cost;
                seg = (int)rows;
            }
        }
    }
    seg = std::max(seg, min_seg);
    const std::vector<int> b = segment_bounds(g, seg, K, h->src.polarization, weight);
    p.n_segs = (int)b.size() - 1;
    p.seg_rows = seg;
    CK(cudaMalloc(&p.d_seg_y0, b.size() * sizeof(int)));
    CK(cudaMemcpy(p.d_seg_y0, b.data(), b.size() * sizeof(int), cudaMemcpyHostToDevice));
    return p;
}

BlockPlan& get_plan(fdtd_handle* h, int K) {
    return plan_for(h, h->plans, K, h->opt_variant, h->opt_weight);
}

int choose_kernel(fdtd_handle* h) {
    if (h->opt_kernel == 1 || h->maps) return 1;   // per-cell materials: per-half-step kernels
    const bool blocked_ok = (h->g.nx % 4 == 0);
    if (h->opt_kernel == 2 && !blocked_ok) {
        h->err = "the blocked kernel needs nx % 4 == 0";
        throw Fail{FDTD_EINVAL};
    }
    return blocked_ok ? 2 : 1;
}

void run_stencil(fdtd_handle* h, int64_t s, int64_t e, int kern) {
    StepArgs a = step_args(h);
    if (kern == 1) {
        for (int64_t n = s; n < e; ++n) {
            launch_naive_step(a, h->ez[h->cur], h->hx[h->cur], h->hy[h->cur], h->psiE[h->cur],
                              h->psiH[h->cur], n, h->stream);
            h->stencil_launches += 1;
            h->total_launches += 3;
        }
        CK(cudaGetLastError());
        return;
    }
    const int Kmax = std::min(h->opt_block, blocked_max_K());
    int64_t n = s;
    while (n < e) {
        const int K = (int)std::min<int64_t>(Kmax, e - n);
        BlockPlan& p = get_plan(h, K);
        BlockedArgs b{};
        b.s = a;
        const int c = h->cur, o = c ^ 1;
        b.ez_in = h->ez[c]; b.hx_in = h->hx[c]; b.hy_in = h->hy[c];
        b.ez_out = h->ez[o]; b.hx_out = h->hx[o]; b.hy_out = h->hy[o];
        b.psiE_in = h->psiE[c]; b.psiH_in = h->psiH[c];
        b.psiE_out = h->psiE[o]; b.psiH_out = h->psiH[o];
        b.seg_y0 = p.d_seg_y0;
        b.n_strips = p.n_strips;
        b.n_tasks = p.n_strips * p.n_segs;
        b.w_int = p.w_int;
        if (!launch_blocked(b, K, h->opt_variant, n, h->stream)) {
            h->err = "no blocked kernel instance for this depth";
            throw Fail{FDTD_EINVAL};
        }
        h->cur = o;
        h->stencil_launches += 1;
        h->total_launches += 1;
        n += K;
    }
    CK(cudaGetLastError());
}

void collect_timing(fdtd_handle* h) {
    for (auto& pr : h->timing_events) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) h->stencil_ms += ms;
        h->event_pool.push_back(pr);
    }
    h->timing_events.clear();
}

std::pair<cudaEvent_t, cudaEvent_t> take_events(fdtd_handle* h) {
    if (!h->event_pool.empty()) {
        auto pr = h->event_pool.back();
        h->event_pool.pop_back();
        return pr;
    }
    std::pair<cudaEvent_t, cudaEvent_t> pr{};
    CK(cudaEventCreate(&pr.first));
    CK(cudaEventCreate(&pr.second));
    return pr;
}

void sync_all(fdtd_handle* h) {
    CK(cudaStreamSynchronize(h->twin_stream));
    CK(cudaStreamSynchronize(h->stream));
    collect_timing(h);
    debug_checks(h);
    if (h->opt_watchdog > 0) {
        int flag = 0;
        CK(cudaMemcpy(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) {
            h->err = "non-finite field values (unstable run)";
            throw Fail{FDTD_EUNSTABLE};
        }
    }
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void free_all(fdtd_handle* h) {
    for (int i = 0; i < 2; ++i) {
        dfree(h->ez[i]); dfree(h->hx[i]); dfree(h->hy[i]);
        dfree(h->psiE[i]); dfree(h->psiH[i]);
    }
    dfree(h->labels); dfree(h->coef); dfree(h->pml_e); dfree(h->pml_h); dfree(h->dft);
    dfree(h->cellcoef); dfree(h->cell_eps); dfree(h->cell_sig);
    for (auto& c : h->ck) dfree(c);
    h->ck.clear();
    for (auto& t : h->adj_tape) dfree(t);
    h->adj_tape.clear();
    for (float*& q : h->adj_state) { dfree(q); q = nullptr; }
    if (h->d_adj_tape_ptrs) { cudaFree(h->d_adj_tape_ptrs); h->d_adj_tape_ptrs = nullptr; }
    dfree(h->tw_ez); dfree(h->tw_hx); dfree(h->tw_psiE); dfree(h->tw_psiH); dfree(h->tw_dft);
    dfree(h->d_flux); dfree(h->d_flag); dfree(h->d_dbg);
    h->guarded.clear();
    dfree(h->d_hinc); dfree(h->d_einc); dfree(h->d_phE); dfree(h->d_phH);
    if (h->h_flux) cudaFreeHost(h->h_flux);
    if (h->h_hinc) cudaFreeHost(h->h_hinc);
    if (h->h_einc) cudaFreeHost(h->h_einc);
    if (h->h_phE) cudaFreeHost(h->h_phE);
    if (h->h_phH) cudaFreeHost(h->h_phH);
    h->h_flux = nullptr; h->h_hinc = nullptr; h->h_einc = nullptr; h->h_phE = nullptr; h->h_phH = nullptr;
    for (auto& p : h->plans) dfree(p.d_seg_y0);
    for (auto& p : h->tape_plans) dfree(p.d_seg_y0);
    for (auto& pr : h->timing_events) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (auto& pr : h->event_pool) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    h->timing_events.clear(); h->event_pool.clear();
    if (h->ev_tab) cudaEventDestroy(h->ev_tab);
    if (h->ev_twin) cudaEventDestroy(h->ev_twin);
    if (h->twin_stream) cudaStreamDestroy(h->twin_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    h->ev_tab = h->ev_twin = nullptr; h->twin_stream = nullptr; h->stream = nullptr;
}

__global__ void k_max_label(const uint8_t* lab, int lpitch, int nx, int ny, int* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < nx) atomicMax(out, (int)lab[(size_t)j * lpitch + i]);
}

}  // namespace fdtd

// --------------------------------------------------------------------------
// incident-wave generator
// --------------------------------------------------------------------------
namespace fdtd {

void IncidentGen::reset(int64_t plan) {
    plan_end = plan;
    m = 0;
    const size_t L = (size_t)(plan / 2 + 16);
    ez.assign(L, 0.0);
    hx.assign(L, 0.0);
}

double IncidentGen::source(double t) const {
    const double f0 = kC0 / lambda0;
    const double w0 = 2.0 * kPi * f0;
    if (kind == 0) {
        const double sigma_f = bw * f0 / (2.0 * std::sqrt(2.0 * std::log(2.0)));
        const double tau = 1.0 / (2.0 * kPi * sigma_f);
        const double t0 = t0_over_tau * tau;
        return std::exp(-((t - t0) * (t - t0)) / (2.0 * tau * tau)) * std::sin(w0 * (t - t0));
    }
    if (kind == 1) {
        const double tr = 10.0 / f0;
        const double ramp = t >= tr ? 1.0 : 0.5 * (1.0 - std::cos(kPi * t / tr));
        return ramp * std::sin(w0 * t);
    }
    return 0.0;
}

void IncidentGen::step(float* hinc, float* einc) {
    *hinc = (float)hx[1];                           // eta0*Hx at edge 1, time m
    const int64_t L = (int64_t)ez.size();
    const int64_t kmax = std::min<int64_t>(std::min<int64_t>(m + 2, plan_end - m + 2), L - 2);
    double* E = ez.data();
    double* Hh = hx.data();
    for (int64_t k = 1; k <= kmax; ++k) E[k] += S * (Hh[k + 1] - Hh[k]);
    E[0] = source(((double)m + 0.5) * dt);
    *einc = (float)E[1];                            // Ez at cell 1, time m+1/2
    for (int64_t k = 1; k <= kmax; ++k) Hh[k] += S * (E[k] - E[k - 1]);
    ++m;
}

}  // namespace fdtd

// --------------------------------------------------------------------------
// C ABI
// --------------------------------------------------------------------------
extern "C" {

static int create_impl(const fdtd_grid* grid, const uint8_t* labels, const fdtd_material* table,
                       int32_t n_labels, const double* eps_map, const double* sig_map,
                       const fdtd_source* source, void* cuda_stream, fdtd_handle** out) {
    if (out) *out = nullptr;
    const bool maps = (eps_map != nullptr);
    if (!grid || !source || !out || (maps ? !sig_map : (!labels || !table))) {
        g_create_err = "fdtd_create: null argument";
        return FDTD_EINVAL;
    }
    fdtd_handle* h = new fdtd_handle();
    try {
        h->g = *grid;
        h->src = *source;
        h->maps = maps;
        if (maps) {
            static const fdtd_material air = {1.0, 0.0};
            table = &air;
            n_labels = 1;
        }
        h->n_labels = n_labels;
        h->table.assign(table, table + n_labels);
        const fdtd_grid& g = h->g;
        REQUIRE(g.nx >= 1 && g.ny >= 8, "grid: need nx >= 1 and ny >= 8");
        REQUIRE((int64_t)g.nx * g.ny < ((int64_t)1 << 31), "grid: more than 2^31 cells");
        REQUIRE(g.dx > 0 && g.dt > 0, "grid: dx and dt must be positive");
        h->S = kC0 * g.dt / g.dx;
        REQUIRE(h->S <= (1.0 / std::sqrt(2.0)) * (1.0 + 1e-12),
                "grid: Courant number c0*dt/dx exceeds the 2D CFL limit 1/sqrt(2)");
        REQUIRE(g.pml_cells >= 0, "grid: pml_cells < 0");
        REQUIRE(g.r_row >= g.pml_cells && g.r_row < g.tfsf_row && g.tfsf_row < g.t_row &&
                    g.t_row + 1 < g.ny - g.pml_cells && g.tfsf_row >= 1,
                "grid: need pml_cells <= r_row < tfsf_row < t_row < ny - pml_cells - 1");
        REQUIRE(g.pml_order >= 0 && g.pml_sigma_max >= 0 && g.pml_kappa_max >= 1 &&
                    g.pml_alpha_max >= 0,
                "grid: CPML parameters out of range");
        REQUIRE(n_labels >= 1 && n_labels <= 256, "table: need 1..256 labels");
        REQUIRE(source->kind >= 0 && source->kind <= 2, "source: kind must be 0, 1 or 2");
        REQUIRE(source->polarization == FDTD_POL_S || source->polarization == FDTD_POL_P,
                "source: polarization must be FDTD_POL_S (0) or FDTD_POL_P (1)");
        const bool pol_p = source->polarization == FDTD_POL_P;
        // default code shape of the blocked kernel: 5 (label-pair table,
        // paired FP32) where the labels fit the pair table, else 2
        h->opt_variant = pair_shape_ok(pol_p, maps, n_labels) ? 5 : 2;
        REQUIRE(!pol_p || (!maps && n_labels <= 16),
                "source: P polarisation needs a label map with at most 16 labels");
        REQUIRE(source->lambda0 > 0, "source: lambda0 must be positive");
        REQUIRE(source->kind != 0 || source->rel_bandwidth > 0,
                "source: rel_bandwidth must be positive");
        h->omega = 2.0 * kPi * kC0 / source->lambda0;

        // S: (C_e, S C_h / eps_r) per label (Sec. 2.3). P: the same per label
        // pair (la << 4 | lb) with eps_r and sigma the means of the two labels,
        // the material of an edge between two cells.
        std::vector<double> leps(n_labels), lsig(n_labels);
        for (int l = 0; l < n_labels; ++l) {
            const double n = table[l].n, k = table[l].k;
            REQUIRE(n > 0 && k >= 0 && n > k, "table: need n > k >= 0 for every label");
            leps[l] = n * n - k * k;
            lsig[l] = 2.0 * h->omega * kEps0 * n * k;
        }
        auto lossy = [&](double eps, double sig) {
            const double beta = sig * g.dt / (2.0 * kEps0 * eps);
            return make_float2((float)((1.0 - beta) / (1.0 + beta)),
                               (float)(h->S / (eps * (1.0 + beta))));
        };
        const int n_coef = pol_p ? 256 : n_labels;
        std::vector<float2> coef(n_coef, make_float2(1.0f, (float)h->S));
        for (int la = 0; la < n_labels; ++la) {
            if (!pol_p) {
                coef[la] = lossy(leps[la], lsig[la]);
                continue;
            }
            for (int lb = 0; lb < n_labels; ++lb)
                coef[(la << 4) | lb] = lossy(0.5 * (leps[la] + leps[lb]), 0.5 * (lsig[la] + lsig[lb]));
        }

        CK(cudaGetDevice(&h->device));
        if (cuda_stream) {
            h->stream = (cudaStream_t)cuda_stream;
        } else {
            CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
            h->own_stream = true;
        }
        CK(cudaStreamCreateWithFlags(&h->twin_stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->ev_tab, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_twin, cudaEventDisableTiming));

        h->pitch = round_up(g.nx, 32);
        h->lpitch = round_up(g.nx, 16);
        const size_t cells = (size_t)h->pitch * g.ny;
        const int P = g.pml_cells;
        const size_t prow = (size_t)std::max(2 * P, 1) * h->pitch;
        for (int i = 0; i < 2; ++i) {
            dalloc(h, &h->ez[i], cells);
            dalloc(h, &h->hx[i], cells);
            dalloc(h, &h->hy[i], cells);
            dalloc(h, &h->psiE[i], prow);
            dalloc(h, &h->psiH[i], prow);
        }
        dalloc(h, &h->labels, (size_t)h->lpitch * g.ny);
        if (!maps)
            CK(cudaMemcpy2DAsync(h->labels, h->lpitch, labels, g.nx, g.nx, g.ny, cudaMemcpyDefault,
                                 h->stream));
        dalloc(h, &h->coef, 256);
        CK(cudaMemcpyAsync(h->coef, coef.data(), n_coef * sizeof(float2), cudaMemcpyHostToDevice,
                           h->stream));
        dalloc(h, &h->dft, (size_t)4 * g.nx);
        dalloc(h, &h->tw_ez, g.ny);
        dalloc(h, &h->tw_hx, g.ny);
        dalloc(h, &h->tw_psiE, std::max(2 * P, 1));
        dalloc(h, &h->tw_psiH, std::max(2 * P, 1));
        dalloc(h, &h->tw_dft, 4);
        dalloc(h, &h->d_flux, 4);
        dalloc(h, &h->d_flag, 4);
        dalloc(h, &h->d_dbg, 1);
        CK(cudaMallocHost(&h->h_flux, 4 * sizeof(double)));

        // CPML tables [3][2P] for Ez rows and Hx rows
        std::vector<float> pe(6 * std::max(P, 1), 0.f), ph(6 * std::max(P, 1), 0.f);
        for (int q = 0; q < 2 * P; ++q) {
            const double de = (q < P) ? (P - q - 0.5) : ((q - P) + 0.5);
            const double dh = (q < P) ? (double)(P - q) : (double)(q - P);
            cpml_coeffs(g, de, &pe[q], &pe[2 * P + q], &pe[4 * P + q]);
            cpml_coeffs(g, dh, &ph[q], &ph[2 * P + q], &ph[4 * P + q]);
        }
        dalloc(h, &h->pml_e, pe.size());
        dalloc(h, &h->pml_h, ph.size());
        CK(cudaMemcpyAsync(h->pml_e, pe.data(), pe.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->pml_h, ph.data(), ph.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));

        // labels: range check on the device, air check of the TF/SF rows
        int* d_max = nullptr;
        CK(cudaMalloc(&d_max, sizeof(int)));
        CK(cudaMemsetAsync(d_max, 0, sizeof(int), h->stream));
        k_max_label<<<dim3((g.nx + 255) / 256, g.ny), 256, 0, h->stream>>>(h->labels, h->lpitch,
                                                                           g.nx, g.ny, d_max);
        int maxl = 0;
        std::vector<uint8_t> rows((size_t)2 * g.nx);
        CK(cudaMemcpyAsync(&maxl, d_max, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpy2DAsync(rows.data(), g.nx, h->labels + (size_t)(g.tfsf_row - 1) * h->lpitch,
                             h->lpitch, g.nx, 2, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        cudaFree(d_max);
        REQUIRE(maxl < n_labels, "labels: a label value is >= n_labels");
        if (source->kind != 2 && !maps) {
            for (uint8_t v : rows)
                REQUIRE(table[v].n == 1.0 && table[v].k == 0.0,
                        "labels: rows tfsf_row-1 and tfsf_row must be air (n = 1, k = 0)");
        }
        if (maps) {
            // per-cell coefficients from eps_r, sigma (FP64 on the host)
            const size_t cells = (size_t)g.nx * g.ny;
            std::vector<double> he(cells), hs(cells);
            CK(cudaMemcpy(he.data(), eps_map, cells * sizeof(double), cudaMemcpyDefault));
            CK(cudaMemcpy(hs.data(), sig_map, cells * sizeof(double), cudaMemcpyDefault));
            std::vector<float2> cc((size_t)h->pitch * g.ny, make_float2(1.0f, (float)h->S));
            for (int j = 0; j < g.ny; ++j)
                for (int i = 0; i < g.nx; ++i) {
                    const double eps = he[(size_t)j * g.nx + i], sig = hs[(size_t)j * g.nx + i];
                    REQUIRE(eps > 0 && sig >= 0 && std::isfinite(eps) && std::isfinite(sig),
                            "maps: need eps_r > 0 and sigma >= 0 in every cell");
                    if (source->kind != 2 && (j == g.tfsf_row - 1 || j == g.tfsf_row))
                        REQUIRE(eps == 1.0 && sig == 0.0,
                                "maps: rows tfsf_row-1 and tfsf_row must be air (eps_r = 1, sigma = 0)");
                    const double beta = sig * g.dt / (2.0 * kEps0 * eps);
                    cc[(size_t)j * h->pitch + i] =
                        make_float2((float)((1.0 - beta) / (1.0 + beta)),
                                    (float)(h->S / (eps * (1.0 + beta))));
                }
            dalloc(h, &h->cellcoef, cc.size());
            CK(cudaMemcpy(h->cellcoef, cc.data(), cc.size() * sizeof(float2), cudaMemcpyHostToDevice));
            dalloc(h, &h->cell_eps, cells);
            dalloc(h, &h->cell_sig, cells);
            CK(cudaMemcpy(h->cell_eps, he.data(), cells * sizeof(double), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(h->cell_sig, hs.data(), cells * sizeof(double), cudaMemcpyHostToDevice));
        }

        IncidentGen gen;
        gen.S = h->S; gen.dt = g.dt; gen.lambda0 = source->lambda0;
        gen.bw = source->rel_bandwidth; gen.t0_over_tau = source->t0_over_tau;
        gen.kind = source->kind;
        h->tables = table_store(gen, h->omega);
        CK(cudaStreamSynchronize(h->stream));
        *out = h;
        return FDTD_OK;
    } catch (const Fail& f) {
        g_create_err = h->err;
        free_all(h);
        delete h;
        return f.code;
    }
}

int fdtd_create(const fdtd_grid* grid, const uint8_t* labels, const fdtd_material* table,
                int32_t n_labels, const fdtd_source* source, void* cuda_stream,
                fdtd_handle** out) {
    if (!labels || !table) {
        if (out) *out = nullptr;
        g_create_err = "fdtd_create: null argument";
        return FDTD_EINVAL;
    }
    return create_impl(grid, labels, table, n_labels, nullptr, nullptr, source, cuda_stream, out);
}

int fdtd_create_maps(const fdtd_grid* grid, const double* eps_r, const double* sigma,
                     const fdtd_source* source, void* cuda_stream, fdtd_handle** out) {
    if (!eps_r || !sigma) {
        if (out) *out = nullptr;
        g_create_err = "fdtd_create_maps: null argument";
        return FDTD_EINVAL;
    }
    return create_impl(grid, nullptr, nullptr, 0, eps_r, sigma, source, cuda_stream, out);
}

int fdtd_run(fdtd_handle* h, int64_t steps) {
    if (!h) return FDTD_EINVAL;
    try {
        REQUIRE(steps >= 0, "fdtd_run: steps < 0");
        if (steps == 0) return FDTD_OK;
        CK(cudaSetDevice(h->device));
        const int kern = choose_kernel(h);
        h->last_kernel = kern;
        const int64_t n_end = h->n + steps;
        ensure_tables(h, n_end);
        TwinArgs tw{};
        tw.ny = h->g.ny; tw.P = h->g.pml_cells; tw.js = h->g.tfsf_row;
        tw.jr = h->g.r_row; tw.jt = h->g.t_row;
        tw.S = (float)h->S; tw.ca = 1.0f; tw.cb = (float)(h->S / 1.0);
        tw.pml_e = h->pml_e; tw.pml_h = h->pml_h;
        tw.hinc = h->d_hinc; tw.einc = h->d_einc; tw.phE = h->d_phE; tw.phH = h->d_phH;
        tw.ez = h->tw_ez; tw.hx = h->tw_hx; tw.psiE = h->tw_psiE; tw.psiH = h->tw_psiH;
        tw.dft = h->tw_dft;
        tw.dbg = h->d_dbg;
        // chunks of whole blocked launches, so only the run's last launch is short
        const int64_t kb = (kern == 2) ? std::max(1, std::min(h->opt_block, blocked_max_K())) : 1;
        const int64_t chunk = std::max<int64_t>(kb, kChunk - kChunk % kb);
        int64_t s = h->n;
        while (s < n_end) {
            const int64_t ce = std::min(n_end, s + chunk);
            produce_tables(h, std::max(ce, h->tab_uploaded));
            tw.n_tab = table_limit(h);
            CK(cudaEventRecord(h->ev_tab, h->stream));
            CK(cudaStreamWaitEvent(h->twin_stream, h->ev_tab, 0));
            launch_twin(tw, s, (int)(ce - s), h->twin_stream);
            h->total_launches += 1;
            std::pair<cudaEvent_t, cudaEvent_t> pr{};
            if (h->opt_timing) {
                pr = take_events(h);
                CK(cudaEventRecord(pr.first, h->stream));
            }
            run_stencil(h, s, ce, kern);
            if (h->opt_timing) {
                CK(cudaEventRecord(pr.second, h->stream));
                h->timing_events.push_back(pr);
            }
            if (h->opt_watchdog > 0 &&
                (ce / h->opt_watchdog != s / h->opt_watchdog || ce == n_end)) {
                launch_check_finite(h->ez[h->cur], h->pitch, h->g.nx, h->g.ny, h->d_flag, h->stream);
                h->total_launches += 1;
            }
            s = ce;
        }
        h->n = n_end;
        CK(cudaEventRecord(h->ev_twin, h->twin_stream));
        CK(cudaStreamWaitEvent(h->stream, h->ev_twin, 0));
        CK(cudaGetLastError());
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

int fdtd_reset(fdtd_handle* h) {
    if (!h) return FDTD_EINVAL;
    try {
        CK(cudaSetDevice(h->device));
        CK(cudaStreamSynchronize(h->twin_stream));
        const fdtd_grid& g = h->g;
        const size_t cells = (size_t)h->pitch * g.ny * sizeof(float);
        const size_t prow = (size_t)std::max(2 * g.pml_cells, 1) * h->pitch * sizeof(float);
        for (int i = 0; i < 2; ++i) {
            CK(cudaMemsetAsync(h->ez[i], 0, cells, h->stream));
            CK(cudaMemsetAsync(h->hx[i], 0, cells, h->stream));
            CK(cudaMemsetAsync(h->hy[i], 0, cells, h->stream));
            CK(cudaMemsetAsync(h->psiE[i], 0, prow, h->stream));
            CK(cudaMemsetAsync(h->psiH[i], 0, prow, h->stream));
        }
        CK(cudaMemsetAsync(h->dft, 0, (size_t)4 * g.nx * sizeof(double2), h->stream));
        CK(cudaMemsetAsync(h->tw_ez, 0, (size_t)g.ny * sizeof(float), h->stream));
        CK(cudaMemsetAsync(h->tw_hx, 0, (size_t)g.ny * sizeof(float), h->stream));
        CK(cudaMemsetAsync(h->tw_psiE, 0, (size_t)std::max(2 * g.pml_cells, 1) * sizeof(float), h->stream));
        CK(cudaMemsetAsync(h->tw_psiH, 0, (size_t)std::max(2 * g.pml_cells, 1) * sizeof(float), h->stream));
        CK(cudaMemsetAsync(h->tw_dft, 0, 4 * sizeof(double2), h->stream));
        CK(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
        CK(cudaEventRecord(h->ev_tab, h->stream));
        CK(cudaStreamWaitEvent(h->twin_stream, h->ev_tab, 0));
        h->n = 0;
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

int fdtd_synchronize(fdtd_handle* h) {
    if (!h) return FDTD_EINVAL;
    try {
        CK(cudaSetDevice(h->device));
        sync_all(h);
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

static int flux_sums(fdtd_handle* h) {
    CK(cudaSetDevice(h->device));
    launch_flux(h->dft, h->tw_dft, h->g.nx, h->d_flux, h->stream);
    h->total_launches += 1;
    CK(cudaMemcpyAsync(h->h_flux, h->d_flux, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    sync_all(h);
    return FDTD_OK;
}

int fdtd_flux(fdtd_handle* h, double* R, double* T) {
    if (!h || !R || !T) return FDTD_EINVAL;
    try {
        flux_sums(h);
        const double sr = h->h_flux[0], st = h->h_flux[1], s0 = h->h_flux[2];
        const double inc = -s0 * h->g.nx;
        *R = sr / inc;
        *T = -st / inc;
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

int fdtd_flux_raw(fdtd_handle* h, double out[3]) {
    if (!h || !out) return FDTD_EINVAL;
    try {
        flux_sums(h);
        const double f = 0.5 * h->g.dx / kEta0;
        out[0] = f * h->h_flux[0];
        out[1] = -f * h->h_flux[1];
        out[2] = -f * h->h_flux[2] * h->g.nx;
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

int fdtd_reset_dft(fdtd_handle* h) {
    if (!h) return FDTD_EINVAL;
    try {
        CK(cudaSetDevice(h->device));
        sync_all(h);
        CK(cudaMemsetAsync(h->dft, 0, (size_t)4 * h->g.nx * sizeof(double2), h->stream));
        CK(cudaMemsetAsync(h->tw_dft, 0, 4 * sizeof(double2), h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

namespace {

// k_y dx of Bloch order m on the 2D lattice:
// sin^2(k_y dx/2) = sin^2(w dt/2)/S^2 - sin^2(pi m/nx); NaN when evanescent.
double bloch_ky(int64_t m, int nx, double S, double wdt) {
    const double a = std::sin(0.5 * wdt) / S;
    const double b = std::sin(kPi * (double)m / (double)nx);
    const double s2 = a * a - b * b;
    if (!(s2 > 0.0) || s2 > 1.0) return std::nan("");
    return 2.0 * std::asin(std::sqrt(s2));
}

}  // namespace

int32_t fdtd_bloch_propagating(const fdtd_handle* h) {
    if (!h) return FDTD_EINVAL;
    const double wdt = h->omega * h->g.dt;
    int32_t M = 0;
    while (2 * (M + 1) + 1 <= h->g.nx && std::isfinite(bloch_ky(M + 1, h->g.nx, h->S, wdt))) ++M;
    return M;
}

int fdtd_bloch_orders(fdtd_handle* h, int32_t m_max, double* out) {
    if (!h || !out) return FDTD_EINVAL;
    double2* d_ord = nullptr;
    try {
        REQUIRE(m_max >= 0 && 2 * (int64_t)m_max + 1 <= h->g.nx,
                "fdtd_bloch_orders: need 0 <= m_max and 2 m_max + 1 <= nx");
        CK(cudaSetDevice(h->device));
        sync_all(h);
        const int n_ord = 2 * m_max + 1;
        CK(cudaMalloc(&d_ord, (size_t)4 * n_ord * sizeof(double2)));
        launch_bloch(h->dft, h->g.nx, m_max, d_ord, h->stream);
        CK(cudaGetLastError());
        h->total_launches += 1;
        std::vector<double2> ord((size_t)4 * n_ord);
        double2 tw[4];
        CK(cudaMemcpyAsync(ord.data(), d_ord, ord.size() * sizeof(double2), cudaMemcpyDeviceToHost,
                           h->stream));
        CK(cudaMemcpyAsync(tw, h->tw_dft, sizeof(tw), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        cudaFree(d_ord);
        d_ord = nullptr;
        // Stored lines (both polarisations, in the device variables): 0 centre
        // field at r_row, 1 averaged edge field at r_row, 2 and 3 at t_row.
        // The flux identities are those of fdtd_flux; the paper's amplitude is
        // the centre field (Ez) for S and the edge field (Ex) for P.
        const bool pol_p = h->src.polarization == FDTD_POL_P;
        const double nx = (double)h->g.nx;
        const double inc = -(tw[2].x * tw[3].x + tw[2].y * tw[3].y) * nx;
        const double2 e_inc = pol_p ? tw[3] : tw[2];
        const double a_inc = e_inc.x * e_inc.x + e_inc.y * e_inc.y;
        const double wdt = h->omega * h->g.dt;
        const double ky0 = bloch_ky(0, h->g.nx, h->S, wdt);
        for (int o = 0; o < n_ord; ++o) {
            const double2 er = ord[o], hr = ord[n_ord + o];
            const double2 et = ord[2 * n_ord + o], ht = ord[3 * n_ord + o];
            const double2 ar = pol_p ? hr : er, at = pol_p ? ht : et;
            const double ky = bloch_ky(o - m_max, h->g.nx, h->S, wdt);
            double w = 0.0;
            if (std::isfinite(ky)) w = pol_p ? std::sin(ky0) / std::sin(ky) : std::sin(ky) / std::sin(ky0);
            double* r = out + (size_t)8 * o;
            r[0] = nx * (er.x * hr.x + er.y * hr.y) / inc;
            r[1] = -nx * (et.x * ht.x + et.y * ht.y) / inc;
            r[2] = (ar.x * ar.x + ar.y * ar.y) / a_inc;
            r[3] = (at.x * at.x + at.y * at.y) / a_inc;
            r[4] = w * r[2];
            r[5] = w * r[3];
            r[6] = w;
            r[7] = ky;
        }
        return FDTD_OK;
    } catch (const Fail& f) {
        if (d_ord) cudaFree(d_ord);
        return f.code;
    }
}

int fdtd_get_dft(fdtd_handle* h, double* out) {
    if (!h || !out) return FDTD_EINVAL;
    try {
        sync_all(h);
        const size_t cnt = (size_t)8 * h->g.nx;
        std::vector<double> tmp(cnt);
        CK(cudaMemcpy(tmp.data(), h->dft, cnt * sizeof(double), cudaMemcpyDeviceToHost));
        // S: rows 1, 3 hold eta0 Hx. P: rows 0, 2 hold eta0 Hz, rows 1, 3 hold -Ex.
        const bool pol_p = h->src.polarization == FDTD_POL_P;
        for (int row = 0; row < 4; ++row) {
            const double sc = pol_p ? ((row & 1) ? -1.0 : 1.0 / kEta0) : ((row & 1) ? 1.0 / kEta0 : 1.0);
            for (size_t i = 0; i < (size_t)2 * h->g.nx; ++i) tmp[(size_t)row * 2 * h->g.nx + i] *= sc;
        }
        CK(cudaMemcpy(out, tmp.data(), cnt * sizeof(double), cudaMemcpyDefault));
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

int fdtd_get_fields(fdtd_handle* h, float* ez, float* hx, float* hy) {
    if (!h) return FDTD_EINVAL;
    try {
        sync_all(h);
        const fdtd_grid& g = h->g;
        const size_t cnt = (size_t)g.nx * g.ny;
        float* tmp = nullptr;
        float* dst[3] = {ez, hx, hy};
        const float* src[3] = {h->ez[h->cur], h->hx[h->cur], h->hy[h->cur]};
        // stored (S) Ez, eta0 Hx, eta0 Hy or (P) eta0 Hz, -Ex, -Ey
        const bool pol_p = h->src.polarization == FDTD_POL_P;
        const float scale[3] = {pol_p ? (float)(1.0 / kEta0) : 1.0f,
                                pol_p ? -1.0f : (float)(1.0 / kEta0),
                                pol_p ? -1.0f : (float)(1.0 / kEta0)};
        for (int f = 0; f < 3; ++f) {
            if (!dst[f]) continue;
            if (is_device_ptr(dst[f])) {
                launch_pack(src[f], h->pitch, g.nx, g.ny, scale[f], dst[f], h->stream);
            } else {
                if (!tmp) CK(cudaMalloc(&tmp, cnt * sizeof(float)));
                launch_pack(src[f], h->pitch, g.nx, g.ny, scale[f], tmp, h->stream);
                CK(cudaMemcpyAsync(dst[f], tmp, cnt * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
            }
            h->total_launches += 1;
        }
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (tmp) cudaFree(tmp);
        CK(e);
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

int fdtd_set_fields(fdtd_handle* h, const float* ez, const float* hx, const float* hy) {
    if (!h) return FDTD_EINVAL;
    try {
        sync_all(h);
        const fdtd_grid& g = h->g;
        const size_t cnt = (size_t)g.nx * g.ny;
        float* tmp = nullptr;
        const float* srcs[3] = {ez, hx, hy};
        float* dsts[3] = {h->ez[h->cur], h->hx[h->cur], h->hy[h->cur]};
        const bool pol_p = h->src.polarization == FDTD_POL_P;
        const float scale[3] = {pol_p ? (float)kEta0 : 1.0f, pol_p ? -1.0f : (float)kEta0,
                                pol_p ? -1.0f : (float)kEta0};
        for (int f = 0; f < 3; ++f) {
            if (!srcs[f]) continue;
            const float* s = srcs[f];
            if (!is_device_ptr(s)) {
                if (!tmp) CK(cudaMalloc(&tmp, cnt * sizeof(float)));
                CK(cudaMemcpyAsync(tmp, s, cnt * sizeof(float), cudaMemcpyHostToDevice, h->stream));
                s = tmp;
            }
            launch_unpack(s, g.nx, g.ny, scale[f], dsts[f], h->pitch, h->stream);
            h->total_launches += 1;
            if (f == 1) CK(cudaMemsetAsync(dsts[1], 0, g.nx * sizeof(float), h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
        if (tmp) cudaFree(tmp);
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

// State layout: header, then the raw device arrays in a fixed order.
struct StateHeader {
    char magic[8];
    int32_t nx, ny, pitch, pml;
    int64_t n;
};

static void state_parts(fdtd_handle* h, std::vector<std::pair<void*, size_t>>& parts) {
    const fdtd_grid& g = h->g;
    const size_t cells = (size_t)h->pitch * g.ny * sizeof(float);
    const size_t prow = (size_t)std::max(2 * g.pml_cells, 1) * h->pitch * sizeof(float);
    const int c = h->cur;
    parts = {{h->ez[c], cells}, {h->hx[c], cells}, {h->hy[c], cells},
             {h->psiE[c], prow}, {h->psiH[c], prow},
             {h->dft, (size_t)4 * g.nx * sizeof(double2)},
             {h->tw_ez, (size_t)g.ny * sizeof(float)}, {h->tw_hx, (size_t)g.ny * sizeof(float)},
             {h->tw_psiE, (size_t)std::max(2 * g.pml_cells, 1) * sizeof(float)},
             {h->tw_psiH, (size_t)std::max(2 * g.pml_cells, 1) * sizeof(float)},
             {h->tw_dft, 4 * sizeof(double2)}};
}

size_t fdtd_state_bytes(const fdtd_handle* hc) {
    if (!hc) return 0;
    fdtd_handle* h = const_cast<fdtd_handle*>(hc);
    std::vector<std::pair<void*, size_t>> parts;
    state_parts(h, parts);
    size_t b = sizeof(StateHeader);
    for (auto& p : parts) b += p.second;
    return b;
}

int fdtd_save_state(fdtd_handle* h, void* buf, size_t bytes) {
    if (!h || !buf) return FDTD_EINVAL;
    try {
        if (bytes != fdtd_state_bytes(h)) {
            h->err = "fdtd_save_state: buffer size differs from fdtd_state_bytes";
            return FDTD_ESTATE;
        }
        sync_all(h);
        StateHeader hd{};
        std::memcpy(hd.magic, "FDTDST01", 8);
        hd.nx = h->g.nx; hd.ny = h->g.ny; hd.pitch = h->pitch; hd.pml = h->g.pml_cells; hd.n = h->n;
        char* p = static_cast<char*>(buf);
        CK(cudaMemcpy(p, &hd, sizeof(hd), cudaMemcpyDefault));
        p += sizeof(hd);
        std::vector<std::pair<void*, size_t>> parts;
        state_parts(h, parts);
        for (auto& pr : parts) {
            CK(cudaMemcpy(p, pr.first, pr.second, cudaMemcpyDefault));
            p += pr.second;
        }
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

int fdtd_load_state(fdtd_handle* h, const void* buf, size_t bytes) {
    if (!h || !buf) return FDTD_EINVAL;
    try {
        if (bytes != fdtd_state_bytes(h)) {
            h->err = "fdtd_load_state: buffer size differs from fdtd_state_bytes";
            return FDTD_ESTATE;
        }
        sync_all(h);
        StateHeader hd{};
        const char* p = static_cast<const char*>(buf);
        CK(cudaMemcpy(&hd, p, sizeof(hd), cudaMemcpyDefault));
        if (std::memcmp(hd.magic, "FDTDST01", 8) != 0 || hd.nx != h->g.nx || hd.ny != h->g.ny ||
            hd.pitch != h->pitch || hd.pml != h->g.pml_cells || hd.n < 0) {
            h->err = "fdtd_load_state: the state belongs to a different grid";
            return FDTD_ESTATE;
        }
        p += sizeof(hd);
        std::vector<std::pair<void*, size_t>> parts;
        state_parts(h, parts);
        for (auto& pr : parts) {
            CK(cudaMemcpy(pr.first, p, pr.second, cudaMemcpyDefault));
            p += pr.second;
        }
        h->n = hd.n;
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

int fdtd_set_option(fdtd_handle* h, int32_t option, int64_t value) {
    if (!h) return FDTD_EINVAL;
    switch (option) {
        case FDTD_OPT_KERNEL:
            if (value < 0 || value > 2) break;
            h->opt_kernel = (int)value;
            return FDTD_OK;
        case FDTD_OPT_BLOCK_STEPS:
            if (value < 1 || value > blocked_max_K()) break;
            h->opt_block = (int)value;
            return FDTD_OK;
        case FDTD_OPT_SEG_ROWS:
            if (value < 0 || value > (1 << 24)) break;
            h->opt_seg = (int)value;
            return FDTD_OK;
        case FDTD_OPT_TIMING:
            h->opt_timing = value ? 1 : 0;
            return FDTD_OK;
        case FDTD_OPT_WATCHDOG:
            if (value < 0) break;
            h->opt_watchdog = value;
            return FDTD_OK;
        case FDTD_OPT_ADJ_BLOCK:
            if (value < 0 || value > 4) break;
            h->opt_adj_block = (int)value;
            return FDTD_OK;
        case FDTD_OPT_DEBUG_TABLE_LIMIT:
#ifdef FDTD_DEBUG_BOUNDS
            if (value < 0) break;
            h->dbg_tab_limit = value;
            return FDTD_OK;
#else
            h->err = "fdtd_set_option: FDTD_OPT_DEBUG_TABLE_LIMIT needs a debug build";
            return FDTD_EINVAL;
#endif
        case FDTD_OPT_DEBUG_POKE_GUARD:
#ifdef FDTD_DEBUG_BOUNDS
            // one byte of the guard band behind the current Ez buffer (a host
            // write into the allocation), which the next check must report
            if (value != 1) break;
            {
                std::pair<void*, size_t> g{nullptr, 0};
                {
                    std::lock_guard<std::mutex> lk(g_guard_mu);
                    auto it = g_guarded.find((void*)h->ez[h->cur]);
                    if (it != g_guarded.end()) g = it->second;
                }
                if (!g.first) break;
                unsigned char* at = static_cast<unsigned char*>(g.first) + kGuardBytes + g.second;
                if (cudaMemsetAsync(at, 0, 1, h->stream) != cudaSuccess) return FDTD_ECUDA;
            }
            return FDTD_OK;
#else
            h->err = "fdtd_set_option: FDTD_OPT_DEBUG_POKE_GUARD needs a debug build";
            return FDTD_EINVAL;
#endif
        case FDTD_OPT_PLAN_WEIGHT:
            if (value < 0 || value > 1000000) break;
            h->opt_weight = value / 1000.0;
            return FDTD_OK;
        case FDTD_OPT_VARIANT:
            if (value < 0 || value > 5 || value == 4) break;   // 4 and 6: adjoint tape shapes
            if (value == 5 && !pair_shape_ok(h->src.polarization == FDTD_POL_P, h->maps,
                                             h->n_labels))
                break;
            h->opt_variant = (int)value;
            return FDTD_OK;
        default:
            break;
    }
    h->err = "fdtd_set_option: unknown option or value out of range";
    return FDTD_EINVAL;
}

int fdtd_get_stats(fdtd_handle* h, fdtd_stats* out) {
    if (!h || !out) return FDTD_EINVAL;
    try {
        sync_all(h);
    } catch (const Fail& f) {
        return f.code;
    }
    out->steps = h->n;
    out->stencil_launches = h->stencil_launches;
    out->total_launches = h->total_launches;
    out->stencil_ms = h->stencil_ms;
    out->kernel = h->last_kernel;
    out->block_steps = h->opt_block;
    int seg = 0;
    for (auto& p : h->plans)
        if (p.K == h->opt_block) seg = p.seg_rows;
    out->seg_rows = seg;
    out->variant = h->opt_variant;
    out->graph = 0;
    return FDTD_OK;
}

int fdtd_plan_segments(const fdtd_grid* g, int32_t seg_rows, int32_t block_steps,
                       int32_t polarization, int32_t* out, int32_t cap) {
    auto fail = [](const char* msg) {
        g_create_err = msg;
        return FDTD_EINVAL;
    };
    if (!g || !out) return fail("fdtd_plan_segments: null argument");
    if (g->nx < 1 || g->ny < 8) return fail("grid: need nx >= 1 and ny >= 8");
    if (g->pml_cells < 0) return fail("grid: pml_cells < 0");
    if (!(g->r_row >= g->pml_cells && g->r_row < g->tfsf_row && g->tfsf_row < g->t_row &&
          g->t_row + 1 < g->ny - g->pml_cells && g->tfsf_row >= 1))
        return fail("grid: need pml_cells <= r_row < tfsf_row < t_row < ny - pml_cells - 1");
    if (block_steps < 1 || block_steps > fdtd::blocked_max_K())
        return fail("fdtd_plan_segments: block_steps must be 1..8");
    if (polarization != FDTD_POL_S && polarization != FDTD_POL_P)
        return fail("fdtd_plan_segments: polarization must be FDTD_POL_S or FDTD_POL_P");
    std::vector<int> b;
    try {
        b = fdtd::segment_bounds(*g, std::max(seg_rows, block_steps + 1), block_steps,
                                 polarization);
    } catch (const std::bad_alloc&) {
        g_create_err = "fdtd_plan_segments: out of host memory";
        return FDTD_ENOMEM;
    }
    if ((int64_t)b.size() > cap) return fail("fdtd_plan_segments: cap below the boundary count");
    std::copy(b.begin(), b.end(), out);
    g_create_err.clear();
    return (int)b.size();
}

const char* fdtd_last_error(const fdtd_handle* h) {
    return h ? h->err.c_str() : g_create_err.c_str();
}

void fdtd_destroy(fdtd_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->twin_stream) cudaStreamSynchronize(h->twin_stream);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

}  // extern "C"
