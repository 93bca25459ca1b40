// Internal declarations of libfdtd: the handle, the incident-wave generator
// and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fdtd.h"
#include "fdtd_device.cuh"

namespace fdtd {

// Echo-free incident lattice (Sec. 2.5), FP64 on the host, H kept as eta0*H.
// Cell 0 is a hard source s(t); the TF/SF line reads Ez at cell 1 (time
// n+1/2) and eta0*Hx at edge 1 (time n). A signal moves at most one cell per
// step, so at step m only cells k <= m+2 can be non-zero, and only cells
// k <= plan_end - m + 2 can still reach cell 1 before step plan_end; the
// update is limited to both bounds, which leaves every recorded value
// exactly as on an unbounded lattice.
struct IncidentGen {
    double S = 0, dt = 0, lambda0 = 0, bw = 0, t0_over_tau = 0;
    int kind = 0;
    int64_t plan_end = 0;  // values are exact for steps < plan_end
    int64_t m = 0;         // next step to produce
    std::vector<double> ez, hx;
    void reset(int64_t plan);
    double source(double t) const;
    void step(float* hinc, float* einc);
};

// Incident and DFT-phase tables shared by all handles with the same source,
// Courant number and time step (e.g. the slices and polarisations of one
// wavelength in a campaign): computed once, copied into each handle's
// pinned buffers. Values are exact for every step below gen.plan_end, so a
// store grown for a longer run serves shorter ones bit for bit. A store lives
// while a handle holds it.
struct TableStore {
    std::mutex mu;
    IncidentGen gen;                  // next step to produce: gen.m
    double omega = 0;
    std::vector<float> hinc, einc;    // steps [0, hinc.size())
    std::vector<double2> phE, phH;
};
std::shared_ptr<TableStore> table_store(const IncidentGen& params, double omega);

// Segment plan of the temporally blocked kernel for one block depth.
struct BlockPlan {
    int K = 0;            // steps per launch
    int halo = 0;         // halo columns per strip side
    int w_int = 0;        // interior columns per strip
    int n_strips = 0;
    int n_segs = 0;
    int seg_rows = 0;
    int variant = -1;
    double weight = 0.0;      // planner weight the plan was cut with (0: default)
    int* d_seg_y0 = nullptr;  // n_segs + 1 row boundaries
};

struct BlockedArgs {
    StepArgs s;
    const float* ez_in; const float* hx_in; const float* hy_in;
    float* ez_out; float* hx_out; float* hy_out;
    const float* psiE_in; const float* psiH_in;
    float* psiE_out; float* psiH_out;
    const int* seg_y0;
    int n_strips, n_tasks, w_int;
    int64_t n_base;               // batch launches: absolute step of the batch start
    // code shapes 4 and 6 (adjoint recompute): for each step n0+k of the
    // launch (k = 0..K-1) the base pointer tape[k] of a [Ez^{n-1/2} | factor
    // of cb in the Ez update] block of tape_f + tape_f floats (pitch layout)
    float* const* tape;
    size_t tape_f;
};

// Arguments of the batched blocked kernel (all simulations in one launch).
struct BatchArgs {
    const BlockedArgs* sims;      // [2][n_sims]: ping-pong orientation 0 and 1
    const int* task_sim;          // simulation of each task
    const int* first_task;        // first task of each simulation
    const int64_t* step_base;     // device: step offset of the current chunk
    int n_sims, n_tasks;
};

struct TwinArgs {
    int64_t n_base;       // batch launches: absolute step of the batch start
    int ny, P, js, jr, jt;
    float S, ca, cb;      // air coefficients
    const float* pml_e; const float* pml_h;
    const float* hinc; const float* einc;
    const double2* phE; const double2* phH;
    float* ez; float* hx; float* psiE; float* psiH;
    double2* dft;         // [4]: Ez(jr), Hx(jr), Ez(jt), Hx(jt)
    int64_t n_tab;        // table entries valid on the device (debug index checks)
    unsigned* dbg;        // error word of the debug index checks (null: none)
};

struct BlockPlan;
// launchers (kernels.cu, blocked.cu)
// tape (S only): the step's gradient factors for the adjoint (k_naive_e)
void launch_naive_step(const StepArgs& a, float* ez, float* hx, float* hy,
                       float* psiE, float* psiH, int64_t n, cudaStream_t st,
                       float* tape = nullptr, size_t tape_f = 0);
void launch_twin(const TwinArgs& a, int64_t n0, int steps, cudaStream_t st);
void launch_flux(const double2* dft, const double2* twin_dft, int nx, double* out,
                 cudaStream_t st);
void launch_pack(const float* src, int pitch, int nx, int ny, float scale, float* dst,
                 cudaStream_t st);
void launch_unpack(const float* src, int nx, int ny, float scale, float* dst, int pitch,
                   cudaStream_t st);
void launch_scale_double(double* p, int64_t n, double scale, cudaStream_t st);
void launch_bloch(const double2* dft, int nx, int m_max, double2* out, cudaStream_t st);
void launch_check_finite(const float* p, int pitch, int nx, int ny, int* flag,
                         cudaStream_t st);
bool launch_blocked(const BlockedArgs& a, int K, int variant, int64_t n0, cudaStream_t st);
bool launch_blocked_batch(const BatchArgs& b, int K, int variant, int step_off, int parity,
                          int pol, cudaStream_t st);
void configure_twin_batch();
void launch_twin_batch(const TwinArgs* tws, int n, int max_ny, int max_P,
                       const int64_t* step_base, int steps, cudaStream_t st);
int blocked_max_K();
// Code shape 5 (paired FP32; for S also the label-pair table): a label map
// with at most 16 labels (P handles always have one).
inline bool pair_shape_ok(bool pol_p, bool maps, int n_labels) {
    (void)pol_p;
    return !maps && n_labels <= 16;
}
int blocked_warps_per_sm(int K, int variant, int pol = 0);

// host helpers shared by the handle, batch and tuning code (api.cu); they
// throw Fail with the handle's error message set
struct Fail {
    int code;
};
StepArgs step_args(fdtd_handle* h);
// table entries that kernels of this handle may read (the debug checks'
// bound); debug builds can lower it to exercise the checks
int64_t table_limit(const fdtd_handle* h);
// Debug builds: every dalloc'd buffer sits between two guard bands of
// kGuardBytes filled with kGuardByte; these check the bands and the index
// error word, and fail with FDTD_EBOUNDS naming what they found.
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;
void debug_checks(fdtd_handle* h);
void launch_guard_check(const unsigned char* p, size_t n, unsigned char want, unsigned* flag,
                        unsigned bit, cudaStream_t st);
void ensure_tables(fdtd_handle* h, int64_t n_end);
void produce_tables(fdtd_handle* h, int64_t upto);
void compute_tables(fdtd_handle* h, int64_t upto);
void upload_tables(fdtd_handle* h, int64_t upto);
int sm_count(fdtd_handle* h);
void sync_all(fdtd_handle* h);
// weight: cost of a general-path iteration in lean iterations (0: the
// measured default of the polarisation)
std::vector<int> segment_bounds(const fdtd_grid& g, int seg, int K, int pol, double weight = 0.0);
BlockPlan& get_plan(fdtd_handle* h, int K);
BlockPlan& plan_for(fdtd_handle* h, std::vector<BlockPlan>& cache, int K, int variant,
                    double weight);
// Planner weights (lean iterations per general-path iteration) of the
// adjoint's kernels (S) where the handle sets none, measured on config 5
// (1000 x 6000, 30 000 steps; backward Gcell-updates/s for recompute /
// reverse weights, with the recompute's skewed two-row trip): 6/8: 133.6,
// 6/10: 133.7, 8/8: 141.8, 8/9: 139.8, 8/10: 141.9, 10/8: 138.9, 10/10:
// 139.1, 12/8: 134.5, 12/10: 134.6; before that trip 12/12 gave 131.5 and
// 8/12 134.9. The recompute (code shapes 4 and 6) stores the gradient
// factors of every row, which makes its lean iterations dearer and the
// general path relatively cheaper.
inline constexpr double kTapeGeneralCost = 8.0;
inline constexpr double kReverseGeneralCost = 10.0;

}  // namespace fdtd

struct fdtd_handle {
    fdtd_grid g{};
    fdtd_source src{};
    int n_labels = 0;
    double S = 0, omega = 0;
    cudaStream_t stream = nullptr, twin_stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int pitch = 0, lpitch = 0;
    // device state
    float* ez[2] = {nullptr, nullptr};
    float* hx[2] = {nullptr, nullptr};
    float* hy[2] = {nullptr, nullptr};
    float* psiE[2] = {nullptr, nullptr};
    float* psiH[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t* labels = nullptr;
    float2* coef = nullptr;
    // per-cell materials (fdtd_create_maps): coefficients and eps_r, sigma
    bool maps = false;
    float2* cellcoef = nullptr;
    double* cell_eps = nullptr;
    double* cell_sig = nullptr;
    std::vector<fdtd_material> table;   // per-label materials (label handles)
    // adjoint: checkpoints of the last fdtd_forward_checkpointed run
    std::vector<float*> ck;             // state at steps 0, every, 2 every, ...
    size_t ck_floats = 0;
    // fdtd_backward's tape (per step of a segment, the gradient factors), the
    // recompute's two state buffers and the device array of tape pointers:
    // kept for the next fdtd_backward of the same size, freed by fdtd_destroy
    std::vector<float*> adj_tape;
    size_t adj_tape_floats = 0;
    float* adj_state[2] = {nullptr, nullptr};
    float** d_adj_tape_ptrs = nullptr;
    int64_t adj_steps = 0;
    int adj_every = 0;
    bool adj_valid = false;
    float* pml_e = nullptr;
    float* pml_h = nullptr;
    double2* dft = nullptr;
    float* tw_ez = nullptr; float* tw_hx = nullptr;
    float* tw_psiE = nullptr; float* tw_psiH = nullptr;
    double2* tw_dft = nullptr;
    double* d_flux = nullptr;
    double* h_flux = nullptr;  // pinned
    int* d_flag = nullptr;
    unsigned* d_dbg = nullptr;   // error word of the debug index checks
    std::vector<void*> guarded;  // debug builds: this handle's guarded buffers
    int64_t dbg_tab_limit = 0;   // debug builds: table entries the checks admit (0: all)
    // incident-wave and phase tables (absolute step index)
    std::shared_ptr<fdtd::TableStore> tables;
    int64_t tab_plan = 0;       // steps the buffers are planned for
    int64_t tab_m = 0;          // entries [0, tab_m) are in the pinned buffers
    int64_t tab_cap = 0;
    float* d_hinc = nullptr; float* d_einc = nullptr;
    double2* d_phE = nullptr; double2* d_phH = nullptr;
    float* h_hinc = nullptr; float* h_einc = nullptr;      // pinned
    double2* h_phE = nullptr; double2* h_phH = nullptr;    // pinned
    int64_t tab_uploaded = 0;   // table entries [0, tab_uploaded) are on the device
    cudaEvent_t ev_tab = nullptr, ev_twin = nullptr;
    // blocked-kernel plans per depth: the forward's and the adjoint recompute's
    std::vector<fdtd::BlockPlan> plans;
    std::vector<fdtd::BlockPlan> tape_plans;
    // options
    int opt_kernel = 0, opt_block = 8, opt_seg = 0, opt_timing = 0, opt_variant = 2;
    double opt_weight = 0.0;    // planner weight of a general-path iteration (0: default)
    int opt_adj_block = 3;      // reverse steps per blocked adjoint launch (0: one per step)
    int64_t opt_watchdog = 0;
    // stats
    int64_t n = 0;
    int64_t stencil_launches = 0, total_launches = 0;
    double stencil_ms = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timing_events;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> event_pool;
    int last_kernel = 0;
    std::string err;
};
