// Batched runs of many independent simulations and the launch-shape
// autotuner.
//
// fdtd_batch_run advances every handle of a batch in lockstep: each launch
// of the blocked kernel covers the union of all simulations' warp tasks
// (strip x segment), so simulations too small to fill the GPU alone share
// the machine; the empty-domain columns of all simulations run as one launch
// on a side stream. Launches are grouped in chunks of an even number of
// launches; a full chunk is captured once into a CUDA graph and replayed,
// with the chunk's starting step read by the kernels from device memory.
//
// The autotuners time candidate (steps per launch K, code shape, segment
// height) with trial launches that read the current state and write only
// the other ping-pong buffers, the CPML carry scratch and a dummy DFT sink,
// so tuning leaves the simulation state untouched.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "fdtd_internal.h"

using namespace fdtd;

struct fdtd_batch {
    std::vector<fdtd_handle*> hs;
    int device = 0;
    cudaStream_t stream = nullptr, side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_in = nullptr;
    int K = 8, variant = 2, seg = 0, timing = 0, use_graph = 1;
    // plan
    bool planned = false;
    int pK = 0, pvar = -1, pseg = -1, seg_used = 0;
    int n_tasks = 0, max_ny = 0, max_P = 0;
    std::vector<int> first_task, n_strips;
    std::vector<int*> d_seg;
    BlockedArgs* d_args = nullptr;
    TwinArgs* d_twin = nullptr;
    int* d_task_sim = nullptr;
    int* d_first_task = nullptr;
    int64_t* d_step_base = nullptr;
    double2* d_dummy = nullptr;
    // captured chunk
    cudaGraphExec_t graph = nullptr;
    int graph_launches = 0;
    // stats
    int64_t steps = 0, launches = 0, total_launches = 0;
    double stencil_ms = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used, ev_pool;
    std::string err;
};

namespace {

#define BCK(call)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            b->err = std::string(#call) + ": " + cudaGetErrorString(e_);            \
            throw Fail{e_ == cudaErrorMemoryAllocation ? FDTD_ENOMEM : FDTD_ECUDA}; \
        }                                                                           \
    } while (0)

__global__ void k_set_i64(int64_t* p, int64_t v) { *p = v; }

// Message of the last failed fdtd_batch_create on this thread.
thread_local std::string g_batch_create_err;
const char* batch_create_error(const char* set) {
    if (set) g_batch_create_err = set;
    return g_batch_create_err.c_str();
}

template <typename T>
void bfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void drop_graph(fdtd_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_launches = 0;
}

void drop_plan(fdtd_batch* b) {
    drop_graph(b);
    for (auto& p : b->d_seg) bfree(p);
    b->d_seg.clear();
    bfree(b->d_args); bfree(b->d_twin); bfree(b->d_task_sim); bfree(b->d_first_task);
    b->planned = false;
}

// Code shape 5 needs every simulation of the batch to allow it.
bool batch_pair_ok(const fdtd_batch* b) {
    for (const auto* h : b->hs)
        if (!pair_shape_ok(h->src.polarization == FDTD_POL_P, h->maps, h->n_labels)) return false;
    return true;
}

// Wave model over the union of the batch: waves x (rows + 2K), each
// simulation cut into ceil(ny / rows) segments so that no task is longer.
int model_seg(fdtd_batch* b, int K, int variant) {
    int per_sm = blocked_warps_per_sm(K, variant, b->hs[0]->src.polarization);
    if (per_sm <= 0) per_sm = 8;
    const int64_t W = (int64_t)sm_count(b->hs[0]) * per_sm;
    const int w_int = 128 - 2 * ((K + 3) / 4 * 4);
    int min_seg = 1, max_ny = 1;
    for (auto* h : b->hs) {
        min_seg = std::max(min_seg, K + 1);
        max_ny = std::max(max_ny, h->g.ny);
    }
    double best = 1e300;
    int seg = max_ny;
    for (int s = min_seg; s <= max_ny; s += std::max(1, s / 64)) {
        int64_t tasks = 0;
        for (auto* h : b->hs) {
            const int strips = (h->g.nx + w_int - 1) / w_int;
            tasks += (int64_t)strips * ((h->g.ny + s - 1) / s);   // no task longer than s rows
        }
        const int64_t waves = (tasks + W - 1) / W;
        const double cost = (double)waves * (s + 2.0 * K);
        if (cost < best - 1e-9) { best = cost; seg = s; }
    }
    return seg;
}

// Build task tables, segment tables and CPML carry scratch for (K, variant, seg).
void build_plan(fdtd_batch* b, int K, int variant, int seg_req) {
    drop_plan(b);
    const int n = (int)b->hs.size();
    const int halo = (K + 3) / 4 * 4;
    const int w_int = 128 - 2 * halo;
    const int seg = seg_req > 0 ? seg_req : model_seg(b, K, variant);
    b->first_task.assign(n + 1, 0);
    b->n_strips.assign(n, 0);
    b->max_ny = 0;
    b->max_P = 0;
    std::vector<int> task_sim;
    for (int s = 0; s < n; ++s) {
        fdtd_handle* h = b->hs[s];
        const int P = h->g.pml_cells;
        // ceil(ny / seg) segments of at most seg rows (the wave model's count)
        const int n_s = std::max(1, (h->g.ny + seg - 1) / seg);
        const int seg_s = (h->g.ny + n_s - 1) / n_s;
        const std::vector<int> bounds =
            segment_bounds(h->g, std::max(seg_s, K + 1), K, h->src.polarization, h->opt_weight);
        int* d = nullptr;
        BCK(cudaMalloc(&d, bounds.size() * sizeof(int)));
        BCK(cudaMemcpy(d, bounds.data(), bounds.size() * sizeof(int), cudaMemcpyHostToDevice));
        b->d_seg.push_back(d);
        const int strips = (h->g.nx + w_int - 1) / w_int;
        const int tasks = strips * ((int)bounds.size() - 1);
        b->n_strips[s] = strips;
        b->first_task[s + 1] = b->first_task[s] + tasks;
        task_sim.insert(task_sim.end(), tasks, s);
        b->max_ny = std::max(b->max_ny, h->g.ny);
        b->max_P = std::max(b->max_P, P);
    }
    b->n_tasks = b->first_task[n];
    BCK(cudaMalloc(&b->d_task_sim, task_sim.size() * sizeof(int)));
    BCK(cudaMemcpy(b->d_task_sim, task_sim.data(), task_sim.size() * sizeof(int), cudaMemcpyHostToDevice));
    BCK(cudaMalloc(&b->d_first_task, (n + 1) * sizeof(int)));
    BCK(cudaMemcpy(b->d_first_task, b->first_task.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice));
    BCK(cudaMalloc(&b->d_args, 2 * n * sizeof(BlockedArgs)));
    BCK(cudaMalloc(&b->d_twin, n * sizeof(TwinArgs)));
    b->pK = K;
    b->pvar = variant;
    b->pseg = seg_req;
    b->seg_used = seg;
    b->planned = true;
}

// Per-simulation kernel arguments for the current state of every handle
// (both ping-pong orientations) and the empty-domain columns.
void upload_args(fdtd_batch* b, bool dummy_dft) {
    const int n = (int)b->hs.size();
    const int halo = (b->pK + 3) / 4 * 4;
    std::vector<BlockedArgs> args(2 * n);
    std::vector<TwinArgs> tw(n);
    for (int s = 0; s < n; ++s) {
        fdtd_handle* h = b->hs[s];
        for (int par = 0; par < 2; ++par) {
            BlockedArgs a{};
            a.s = step_args(h);
            if (dummy_dft) a.s.dft = b->d_dummy;
            const int c = h->cur ^ par, o = c ^ 1;
            a.ez_in = h->ez[c]; a.hx_in = h->hx[c]; a.hy_in = h->hy[c];
            a.ez_out = h->ez[o]; a.hx_out = h->hx[o]; a.hy_out = h->hy[o];
            a.psiE_in = h->psiE[c]; a.psiH_in = h->psiH[c];
            a.psiE_out = h->psiE[o]; a.psiH_out = h->psiH[o];
            a.seg_y0 = b->d_seg[s];
            a.n_strips = b->n_strips[s];
            a.n_tasks = b->first_task[s + 1] - b->first_task[s];
            a.w_int = 128 - 2 * halo;
            a.n_base = h->n;
            args[(size_t)par * n + s] = a;
        }
        TwinArgs t{};
        t.n_base = h->n;
        t.ny = h->g.ny; t.P = h->g.pml_cells; t.js = h->g.tfsf_row;
        t.jr = h->g.r_row; t.jt = h->g.t_row;
        t.S = (float)h->S; t.ca = 1.0f; t.cb = (float)(h->S / 1.0);
        t.pml_e = h->pml_e; t.pml_h = h->pml_h;
        t.hinc = h->d_hinc; t.einc = h->d_einc; t.phE = h->d_phE; t.phH = h->d_phH;
        t.ez = h->tw_ez; t.hx = h->tw_hx; t.psiE = h->tw_psiE; t.psiH = h->tw_psiH;
        t.dft = h->tw_dft;
        t.n_tab = table_limit(h);
        t.dbg = h->d_dbg;
        tw[s] = t;
    }
    BCK(cudaMemcpyAsync(b->d_args, args.data(), args.size() * sizeof(BlockedArgs),
                        cudaMemcpyHostToDevice, b->stream));
    BCK(cudaMemcpyAsync(b->d_twin, tw.data(), tw.size() * sizeof(TwinArgs), cudaMemcpyHostToDevice,
                        b->stream));
    BCK(cudaStreamSynchronize(b->stream));   // host vectors go out of scope
}

BatchArgs batch_args(fdtd_batch* b) {
    BatchArgs a{};
    a.sims = b->d_args;
    a.task_sim = b->d_task_sim;
    a.first_task = b->d_first_task;
    a.step_base = b->d_step_base;
    a.n_sims = (int)b->hs.size();
    a.n_tasks = b->n_tasks;
    return a;
}

int launches_per_chunk(int K) { return 2 * std::max(1, 512 / K); }

// Launches of one chunk: `nl` blocked launches of depth K starting at step
// offset 0 of the chunk (parity 0), a trailing launch of depth rem if > 0,
// and the empty-domain columns on the side stream.
void enqueue_chunk(fdtd_batch* b, int nl, int rem, int chunk_steps) {
    const BatchArgs a = batch_args(b);
    const int pol = b->hs[0]->src.polarization;
    BCK(cudaEventRecord(b->ev_fork, b->stream));
    BCK(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
    launch_twin_batch(b->d_twin, (int)b->hs.size(), b->max_ny, b->max_P, b->d_step_base,
                      chunk_steps, b->side);
    for (int j = 0; j < nl; ++j)
        launch_blocked_batch(a, b->pK, b->pvar, j * b->pK, j & 1, pol, b->stream);
    if (rem > 0) launch_blocked_batch(a, rem, b->pvar, nl * b->pK, nl & 1, pol, b->stream);
    BCK(cudaEventRecord(b->ev_join, b->side));
    BCK(cudaStreamWaitEvent(b->stream, b->ev_join, 0));
}

std::pair<cudaEvent_t, cudaEvent_t> take_pair(fdtd_batch* b) {
    if (!b->ev_pool.empty()) {
        auto p = b->ev_pool.back();
        b->ev_pool.pop_back();
        return p;
    }
    std::pair<cudaEvent_t, cudaEvent_t> p{};
    BCK(cudaEventCreate(&p.first));
    BCK(cudaEventCreate(&p.second));
    return p;
}

void collect(fdtd_batch* b) {
    for (auto& p : b->ev_used) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) b->stencil_ms += ms;
        b->ev_pool.push_back(p);
    }
    b->ev_used.clear();
}

double time_trial(fdtd_batch* b, int K, int variant, int seg, int trials) {
    build_plan(b, K, variant, seg);
    upload_args(b, true);
    BCK(cudaMemsetAsync(b->d_step_base, 0, sizeof(int64_t), b->stream));
    const BatchArgs a = batch_args(b);
    const int pol = b->hs[0]->src.polarization;
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    launch_blocked_batch(a, K, variant, 0, 0, pol, b->stream);            // warm-up
    BCK(cudaEventRecord(e0, b->stream));
    for (int t = 0; t < trials; ++t) launch_blocked_batch(a, K, variant, 0, 0, pol, b->stream);
    BCK(cudaEventRecord(e1, b->stream));
    BCK(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BCK(cudaGetLastError());
    double cells = 0;
    for (auto* h : b->hs) cells += (double)h->g.nx * h->g.ny;
    return cells * K * trials / (ms * 1e-3);    // cell-updates per second
}

int batch_tune(fdtd_batch* b, int trials) {
    // the trial launches read the tables of the next K steps
    for (auto* h : b->hs) {
        ensure_tables(h, h->n + blocked_max_K());
        produce_tables(h, std::max(h->n + blocked_max_K(), h->tab_uploaded));
        BCK(cudaEventRecord(h->ev_tab, h->stream));
        BCK(cudaStreamWaitEvent(b->stream, h->ev_tab, 0));
    }
    if (!b->d_dummy) {
        int nx = 0;
        for (auto* h : b->hs) nx = std::max(nx, h->g.nx);
        BCK(cudaMalloc(&b->d_dummy, (size_t)4 * nx * sizeof(double2)));
    }
    double best = -1;
    int bK = b->K, bv = b->variant, bs = 0;
    for (int K : {8, 7, 6}) {
        for (int v : {0, 1, 2, 3, 5}) {
            if (K == 8 && v == 1) continue;          // exceeds the register file at K = 8
            if (b->hs[0]->src.polarization && v < 2) continue;   // P: shapes 2, 3 and 5
            if (v == 5 && !batch_pair_ok(b)) continue;
            const int s0 = model_seg(b, K, v);
            for (int f : {-1, 0, 1}) {
                const int seg = f < 0 ? std::max(1, (s0 * 2) / 3) : (f > 0 ? (s0 * 3) / 2 : s0);
                const double r = time_trial(b, K, v, seg, trials);
                if (r > best) { best = r; bK = K; bv = v; bs = seg; }
            }
        }
    }
    b->K = bK;
    b->variant = bv;
    b->seg = bs;
    drop_plan(b);
    return FDTD_OK;
}

}  // namespace

extern "C" {

int fdtd_batch_create(fdtd_handle* const* hs, int32_t n, fdtd_batch** out) {
    if (out) *out = nullptr;
    if (!hs || n < 1 || !out) return FDTD_EINVAL;
    fdtd_batch* b = new fdtd_batch();
    try {
        for (int i = 0; i < n; ++i) {
            if (!hs[i]) {
                b->err = "fdtd_batch_create: null handle";
                throw Fail{FDTD_EINVAL};
            }
            for (int j = 0; j < i; ++j)
                if (hs[j] == hs[i]) {
                    b->err = "fdtd_batch_create: a handle appears twice";
                    throw Fail{FDTD_EINVAL};
                }
            if (hs[i]->g.nx % 4 != 0) {
                b->err = "fdtd_batch_create: every simulation needs nx % 4 == 0";
                throw Fail{FDTD_EINVAL};
            }
            if (hs[i]->device != hs[0]->device) {
                b->err = "fdtd_batch_create: handles on different devices";
                throw Fail{FDTD_EINVAL};
            }
            if (hs[i]->src.polarization != hs[0]->src.polarization) {
                b->err = "fdtd_batch_create: all handles of a batch need one polarisation";
                throw Fail{FDTD_EINVAL};
            }
            b->hs.push_back(hs[i]);
        }
        b->device = hs[0]->device;
        BCK(cudaSetDevice(b->device));
        b->stream = hs[0]->stream;
        BCK(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
        BCK(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
        BCK(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
        BCK(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
        BCK(cudaMalloc(&b->d_step_base, sizeof(int64_t)));
        configure_twin_batch();
        b->K = std::min(hs[0]->opt_block, blocked_max_K());
        b->variant = hs[0]->opt_variant;
        if (b->variant == 5 && !batch_pair_ok(b)) b->variant = 2;
        *out = b;
        return FDTD_OK;
    } catch (const Fail& f) {
        batch_create_error(b->err.c_str());
        if (b->side) cudaStreamDestroy(b->side);
        if (b->ev_fork) cudaEventDestroy(b->ev_fork);
        if (b->ev_join) cudaEventDestroy(b->ev_join);
        if (b->ev_in) cudaEventDestroy(b->ev_in);
        bfree(b->d_step_base);
        delete b;
        return f.code;
    }
}

int fdtd_batch_set_option(fdtd_batch* b, int32_t option, int64_t value) {
    if (!b) return FDTD_EINVAL;
    switch (option) {
        case FDTD_OPT_BLOCK_STEPS:
            if (value < 1 || value > blocked_max_K()) break;
            b->K = (int)value;
            return FDTD_OK;
        case FDTD_OPT_SEG_ROWS:
            if (value < 0 || value > (1 << 24)) break;
            b->seg = (int)value;
            return FDTD_OK;
        case FDTD_OPT_VARIANT:
            if (value < 0 || value > 5 || value == 4) break;
            if (value == 5 && !batch_pair_ok(b)) break;
            b->variant = (int)value;
            return FDTD_OK;
        case FDTD_OPT_TIMING:
            b->timing = value ? 1 : 0;
            return FDTD_OK;
        case FDTD_OPT_GRAPH:
            b->use_graph = value ? 1 : 0;
            return FDTD_OK;
        default:
            break;
    }
    b->err = "fdtd_batch_set_option: unknown option or value out of range";
    return FDTD_EINVAL;
}

int fdtd_batch_autotune(fdtd_batch* b, int32_t trial_launches) {
    if (!b) return FDTD_EINVAL;
    try {
        BCK(cudaSetDevice(b->device));
        for (auto* h : b->hs) {
            BCK(cudaEventRecord(b->ev_in, h->stream));
            BCK(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
        }
        batch_tune(b, std::max(1, (int)trial_launches));
        BCK(cudaStreamSynchronize(b->stream));
        return FDTD_OK;
    } catch (const Fail& f) {
        for (auto* h : b->hs)
            if (!h->err.empty() && b->err.empty()) b->err = h->err;
        return f.code;
    }
}

int fdtd_batch_run(fdtd_batch* b, int64_t steps) {
    if (!b) return FDTD_EINVAL;
    try {
        if (steps < 0) {
            b->err = "fdtd_batch_run: steps < 0";
            return FDTD_EINVAL;
        }
        if (steps == 0) return FDTD_OK;
        BCK(cudaSetDevice(b->device));
        const int K = std::min(b->K, blocked_max_K());
        const int var = (K == 8 && b->variant == 1) ? 0 : b->variant;
        if (!b->planned || b->pK != K || b->pvar != var || b->pseg != b->seg) {
            BCK(cudaStreamSynchronize(b->stream));
            build_plan(b, K, var, b->seg);
        }
        // earlier work of every handle, then the tables of this run
        for (auto* h : b->hs) {
            BCK(cudaEventRecord(b->ev_in, h->stream));
            BCK(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
            BCK(cudaEventRecord(b->ev_in, h->twin_stream));
            BCK(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
            ensure_tables(h, h->n + steps);
        }
        upload_args(b, false);
        const int nl_full = launches_per_chunk(K);
        const int64_t chunk = (int64_t)nl_full * K;
        int64_t s = 0;
        const int n_threads = (int)std::max<unsigned>(
            1u, std::min<unsigned>((unsigned)b->hs.size(), std::thread::hardware_concurrency()));
        while (s < steps) {
            const int64_t ce = std::min(steps, s + chunk);
            // host-side incident tables of every handle, in parallel
            {
                std::vector<std::thread> pool;
                for (int t = 0; t < n_threads; ++t)
                    pool.emplace_back([&, t]() {
                        for (size_t q = t; q < b->hs.size(); q += n_threads) {
                            fdtd_handle* h = b->hs[q];
                            compute_tables(h, std::max(h->n + ce, h->tab_uploaded));
                        }
                    });
                for (auto& th : pool) th.join();
            }
            for (auto* h : b->hs) {
                upload_tables(h, std::max(h->n + ce, h->tab_uploaded));
                BCK(cudaEventRecord(h->ev_tab, h->stream));
                BCK(cudaStreamWaitEvent(b->stream, h->ev_tab, 0));
            }
            k_set_i64<<<1, 1, 0, b->stream>>>(b->d_step_base, s);
            std::pair<cudaEvent_t, cudaEvent_t> pr{};
            if (b->timing) {
                pr = take_pair(b);
                BCK(cudaEventRecord(pr.first, b->stream));
            }
            const int64_t len = ce - s;
            const int nl = (int)(len / K);
            const int rem = (int)(len % K);
            if (len == chunk && b->use_graph) {
                if (!b->graph) {
                    cudaGraph_t g = nullptr;
                    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                    enqueue_chunk(b, nl, 0, (int)len);
                    BCK(cudaStreamEndCapture(b->stream, &g));
                    const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
                    cudaGraphDestroy(g);
                    if (e != cudaSuccess) {
                        b->graph = nullptr;
                        b->use_graph = 0;
                        cudaGetLastError();
                    } else {
                        b->graph_launches = nl;
                    }
                }
                if (b->graph) BCK(cudaGraphLaunch(b->graph, b->stream));
                else enqueue_chunk(b, nl, 0, (int)len);
            } else {
                enqueue_chunk(b, nl, rem, (int)len);
            }
            b->launches += nl + (rem > 0);
            b->total_launches += nl + (rem > 0) + 2;
            if (b->timing) {
                BCK(cudaEventRecord(pr.second, b->stream));
                b->ev_used.push_back(pr);
            }
            s = ce;
        }
        BCK(cudaGetLastError());
        const int64_t total_launches = (steps / chunk) * nl_full + ((steps % chunk) / K) +
                                       (((steps % chunk) % K) > 0);
        BCK(cudaEventRecord(b->ev_in, b->stream));
        for (auto* h : b->hs) {
            h->n += steps;
            if (total_launches & 1) h->cur ^= 1;
            BCK(cudaStreamWaitEvent(h->stream, b->ev_in, 0));
            BCK(cudaStreamWaitEvent(h->twin_stream, b->ev_in, 0));
        }
        b->steps += steps;
        return FDTD_OK;
    } catch (const Fail& f) {
        for (auto* h : b->hs)
            if (!h->err.empty() && b->err.empty()) b->err = h->err;
        return f.code;
    }
}

int fdtd_batch_get_stats(fdtd_batch* b, fdtd_stats* out) {
    if (!b || !out) return FDTD_EINVAL;
    if (cudaSetDevice(b->device) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess) {
        b->err = "fdtd_batch_get_stats: stream synchronisation failed";
        return FDTD_ECUDA;
    }
    collect(b);
    out->steps = b->steps;
    out->stencil_launches = b->launches;
    out->total_launches = b->total_launches;
    out->stencil_ms = b->stencil_ms;
    out->kernel = 2;
    out->block_steps = b->planned ? b->pK : b->K;
    out->seg_rows = b->planned ? b->seg_used : b->seg;
    out->variant = b->variant;
    out->graph = b->graph ? 1 : 0;
    return FDTD_OK;
}

const char* fdtd_batch_last_error(const fdtd_batch* b) {
    return b ? b->err.c_str() : batch_create_error(nullptr);
}

void fdtd_batch_destroy(fdtd_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->side) cudaStreamSynchronize(b->side);
    drop_plan(b);
    bfree(b->d_step_base);
    bfree(b->d_dummy);
    for (auto& p : b->ev_used) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
    for (auto& p : b->ev_pool) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->side) cudaStreamDestroy(b->side);
    delete b;
}

// Single-handle autotuning: a batch of one, with its choice stored on the
// handle and remembered per (nx, ny, pml_cells, polarisation, device) for
// later handles.
int fdtd_autotune(fdtd_handle* h, int32_t trial_launches) {
    if (!h) return FDTD_EINVAL;
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int>, std::tuple<int, int, int>> cache;
    const auto key = std::make_tuple(h->g.nx, h->g.ny, h->g.pml_cells, h->src.polarization,
                                     h->device);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            h->opt_block = std::get<0>(it->second);
            h->opt_variant = std::get<1>(it->second);
            h->opt_seg = std::get<2>(it->second);
            return FDTD_OK;
        }
    }
    if (h->g.nx % 4 != 0) return FDTD_OK;           // the per-half-step kernels have no knobs
    fdtd_batch* b = nullptr;
    int rc = fdtd_batch_create(&h, 1, &b);
    if (rc != FDTD_OK) return rc;
    rc = fdtd_batch_autotune(b, trial_launches);
    if (rc == FDTD_OK) {
        h->opt_block = b->K;
        h->opt_variant = b->variant;
        h->opt_seg = b->seg;
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = std::make_tuple(b->K, b->variant, b->seg);
    } else {
        h->err = b->err;
    }
    fdtd_batch_destroy(b);
    return rc;
}

}  // extern "C"
