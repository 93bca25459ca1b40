// fdtd_blocked_advance_noalloc: the temporally blocked stencil for callers
// that cannot allocate device memory.
//
// Some callers may not call cudaMalloc where they step the fields: a plug-in
// that must stay inside a fixed device-memory budget owned by its host
// framework, or a process whose device memory is managed by another
// runtime's allocator (a framework's caching allocator that already holds
// the GPU's memory). fdtd_create/fdtd_run allocate (state, tables, plans),
// so this entry point takes every input and output buffer from the caller
// and keeps its own scratch (the segment table, the coefficient and CPML
// tables, zeroed source tables and a sink for monitor sums) in one
// file-scope __device__ array of kScratchBytes. Every GPU that loads the
// library holds that array until the process exits. A call launches two
// kernels on the caller's stream: one that stages the host-computed tables
// (passed by value as its parameters) into the array, and the blocked
// stencil (code shape 5 for at most 16 labels, else 2).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "fdtd_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;   // 8 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kMaxPml = 64;
constexpr int kMaxSegs = 4096;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (in host code the symbol is only a stand-in).
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Host-computed tables of one call, passed by value as kernel parameters
// (about 22 KB, inside the 32 764-byte parameter limit).
struct Staged {
    float2 coef[256];
    float pe[6 * kMaxPml], ph[6 * kMaxPml];
    int bounds[kMaxSegs + 1];
    int n_coef, n_bounds;
};
static_assert(sizeof(Staged) < 32000, "staging parameters exceed the kernel parameter limit");

__global__ void k_stage(const Staged t, float2* coef, float* pe, float* ph, int* seg,
                        unsigned char* zero_tab, size_t zero_tab_bytes, double2* dft,
                        size_t n_dft) {
    const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t st = (size_t)gridDim.x * blockDim.x;
    for (size_t i = i0; i < (size_t)t.n_coef; i += st) coef[i] = t.coef[i];
    for (size_t i = i0; i < (size_t)(6 * kMaxPml); i += st) {
        pe[i] = t.pe[i];
        ph[i] = t.ph[i];
    }
    for (size_t i = i0; i < (size_t)t.n_bounds; i += st) seg[i] = t.bounds[i];
    for (size_t i = i0; i < zero_tab_bytes; i += st) zero_tab[i] = 0;
    for (size_t i = i0; i < n_dft; i += st) dft[i] = make_double2(0.0, 0.0);
}

constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

int fail(char* err, size_t err_len, int code, const char* msg) {
    if (err && err_len) std::snprintf(err, err_len, "%s", msg);
    return code;
}

}  // namespace

extern "C" int fdtd_blocked_advance_noalloc(const fdtd_grid* grid, const uint8_t* labels,
                                            const fdtd_material* table, int32_t n_labels,
                                            double lambda0, const float* const* in,
                                            float* const* out, int32_t steps,
                                            void* cuda_stream, char* err, size_t err_len) {
    using namespace fdtd;
    char msg[192];
    if (!grid || !labels || !table || !in || !out)
        return fail(err, err_len, FDTD_EINVAL, "null argument");
    const fdtd_grid& g = *grid;
    const int P = g.pml_cells;
    if (steps < 1 || steps > blocked_max_K())
        return fail(err, err_len, FDTD_EINVAL, "steps must be 1..8 per call");
    if (g.nx < 4 || g.nx % 4 != 0 || g.ny < 8)
        return fail(err, err_len, FDTD_EINVAL, "need nx >= 4, nx % 4 == 0 and ny >= 8");
    if (!(g.dx > 0 && g.dt > 0) || kC0 * g.dt / g.dx > (1.0 / std::sqrt(2.0)) * (1.0 + 1e-12))
        return fail(err, err_len, FDTD_EINVAL, "Courant number exceeds the 2D CFL limit 1/sqrt(2)");
    if (P < 0 || P > kMaxPml || !(g.r_row >= P && g.r_row < g.tfsf_row && g.tfsf_row < g.t_row &&
                                  g.t_row + 1 < g.ny - P && g.tfsf_row >= 1))
        return fail(err, err_len, FDTD_EINVAL, "row layout or pml_cells (max 64) out of range");
    if (!(g.pml_order >= 0 && g.pml_sigma_max >= 0 && g.pml_kappa_max >= 1 && g.pml_alpha_max >= 0))
        return fail(err, err_len, FDTD_EINVAL, "CPML parameters out of range");
    if (n_labels < 1 || n_labels > 256 || !(lambda0 > 0))
        return fail(err, err_len, FDTD_EINVAL, "need 1..256 labels and lambda0 > 0");
    if (reinterpret_cast<uintptr_t>(labels) % 4 != 0)
        return fail(err, err_len, FDTD_EINVAL, "labels must be 4-byte aligned");
    for (int f = 0; f < 5; ++f) {
        if (!in[f] || !out[f]) return fail(err, err_len, FDTD_EINVAL, "null field buffer");
        if (reinterpret_cast<uintptr_t>(in[f]) % 16 != 0 ||
            reinterpret_cast<uintptr_t>(out[f]) % 16 != 0)
            return fail(err, err_len, FDTD_EINVAL, "field buffers must be 16-byte aligned");
        for (int q = 0; q < 5; ++q)
            if ((const void*)in[f] == (const void*)out[q])
                return fail(err, err_len, FDTD_EINVAL, "output buffers must not alias inputs");
    }

    // scratch layout (256-byte aligned parts)
    const int K = steps;
    const int halo = (K + 3) / 4 * 4;
    const int w_int = 128 - 2 * halo;
    const int n_strips = (g.nx + w_int - 1) / w_int;
    const size_t off_coef = 0;
    const size_t off_pml_e = align256(off_coef + 256 * sizeof(float2));
    const size_t off_pml_h = align256(off_pml_e + 6 * kMaxPml * sizeof(float));
    const size_t off_tab = align256(off_pml_h + 6 * kMaxPml * sizeof(float));
    const size_t tab_bytes = 8 * (2 * sizeof(float) + 2 * sizeof(double2));
    const size_t off_seg = align256(off_tab + tab_bytes);
    const size_t off_dft = align256(off_seg + (kMaxSegs + 1) * sizeof(int));
    const size_t need = off_dft + (size_t)4 * g.nx * sizeof(double2);
    if (need > kScratchBytes) {
        std::snprintf(msg, sizeof msg,
                      "grid needs %zu bytes of scratch, more than the %zu-byte maximum "
                      "(about nx <= 130000)", need, kScratchBytes);
        return fail(err, err_len, FDTD_EINVAL, msg);
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(err, err_len, FDTD_ECUDA, "no usable current device");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            const cudaError_t e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                std::snprintf(msg, sizeof msg, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return fail(err, err_len, FDTD_ECUDA, msg);
            }
        }
        base = g_addr[dev];
    }
    unsigned char* sb = static_cast<unsigned char*>(base);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // host-side tables on the stack (FP64 arithmetic rounded to FP32), in
    // the parameter block of the staging launch
    const double mu0 = 4.0e-7 * kPi;
    const double eps0 = 1.0 / (mu0 * kC0 * kC0);
    const double S = kC0 * g.dt / g.dx;
    const double omega = 2.0 * kPi * kC0 / lambda0;
    Staged tab{};
    float2* coef = tab.coef;
    for (int l = 0; l < n_labels; ++l) {
        const double n = table[l].n, k = table[l].k;
        if (!(n > 0 && k >= 0 && n > k))
            return fail(err, err_len, FDTD_EINVAL, "table: need n > k >= 0 for every label");
        const double eps = n * n - k * k;
        const double sig = 2.0 * omega * eps0 * n * k;
        const double beta = sig * g.dt / (2.0 * eps0 * eps);
        coef[l] = make_float2((float)((1.0 - beta) / (1.0 + beta)), (float)(S / (eps * (1.0 + beta))));
    }
    float* pe = tab.pe;
    float* ph = tab.ph;
    auto prof = [&](double depth, float* b, float* c, float* ik) {
        const double x = depth / (double)P;
        const double xm = std::pow(x, g.pml_order);
        const double sig = g.pml_sigma_max * xm;
        const double kap = 1.0 + (g.pml_kappa_max - 1.0) * xm;
        const double alp = g.pml_alpha_max * (1.0 - x);
        const double bb = std::exp(-(sig / kap + alp) * g.dt / eps0);
        const double den = sig * kap + kap * kap * alp;
        const double cc = (sig > 0.0 && den > 0.0) ? sig * (bb - 1.0) / den : 0.0;
        *b = (float)bb;
        *c = (float)cc;
        *ik = (float)(1.0 / kap);
    };
    for (int q = 0; q < 2 * P; ++q) {
        const double de = (q < P) ? (P - q - 0.5) : ((q - P) + 0.5);
        const double dh = (q < P) ? (double)(P - q) : (double)(q - P);
        prof(de, &pe[q], &pe[2 * P + q], &pe[4 * P + q]);
        prof(dh, &ph[q], &ph[2 * P + q], &ph[4 * P + q]);
    }

    // segment plan: the same wave-count model as the handle path
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 148;
    // code shape 5 (label-pair table, paired FP32) where the labels fit it,
    // else 2, as for handles
    const int shape = pair_shape_ok(false, false, n_labels) ? 5 : 2;
    int per_sm = blocked_warps_per_sm(K, shape);
    if (per_sm <= 0) per_sm = 8;
    const int64_t W = (int64_t)sms * per_sm;
    const int min_seg = P + K + 1;
    int seg = g.ny;
    double best = 1e300;
    for (int n = 1; n <= std::max(1, g.ny / min_seg) && n <= kMaxSegs; ++n) {
        const int64_t waves = ((int64_t)n * n_strips + W - 1) / W;
        const double rows = std::ceil((double)g.ny / n);
        const double cost = (double)waves * (rows + 2.0 * K);
        if (cost < best - 1e-9) { best = cost; seg = (int)rows; }
    }
    seg = std::max(seg, min_seg);
    int* bounds = tab.bounds;
    int nb = 0;
    bounds[nb++] = 0;
    for (int pos = seg; pos < g.ny && nb < kMaxSegs; pos += seg) {
        if (pos == g.r_row + 1 || pos == g.t_row + 1) ++pos;
        if (g.ny - pos < min_seg) break;
        bounds[nb++] = pos;
    }
    bounds[nb++] = g.ny;

    // The tables travel by value as the parameters of one staging launch,
    // which copies them into the scratch array and clears the zeroed parts:
    // nothing is read from host memory after this call returns.
    tab.n_coef = n_labels;
    tab.n_bounds = nb;
    float2* d_coef = reinterpret_cast<float2*>(sb + off_coef);
    float* d_pe = reinterpret_cast<float*>(sb + off_pml_e);
    float* d_ph = reinterpret_cast<float*>(sb + off_pml_h);
    int* d_seg = reinterpret_cast<int*>(sb + off_seg);
    unsigned char* d_tab = sb + off_tab;
    double2* d_dft = reinterpret_cast<double2*>(sb + off_dft);
    k_stage<<<32, 256, 0, st>>>(tab, d_coef, d_pe, d_ph, d_seg, d_tab, tab_bytes, d_dft,
                                (size_t)4 * g.nx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        std::snprintf(msg, sizeof msg, "staging the tables: %s", cudaGetErrorString(e));
        return fail(err, err_len, FDTD_ECUDA, msg);
    }

    BlockedArgs a{};
    a.s.nx = g.nx; a.s.ny = g.ny; a.s.pitch = g.nx; a.s.lpitch = g.nx; a.s.P = P;
    a.s.js = g.tfsf_row; a.s.jr = g.r_row; a.s.jt = g.t_row; a.s.n_labels = n_labels;
    a.s.S = (float)S;
    a.s.labels = labels;
    a.s.coef = reinterpret_cast<const float2*>(sb + off_coef);
    a.s.pml_e = reinterpret_cast<const float*>(sb + off_pml_e);
    a.s.pml_h = reinterpret_cast<const float*>(sb + off_pml_h);
    a.s.hinc = reinterpret_cast<const float*>(sb + off_tab);
    a.s.einc = reinterpret_cast<const float*>(sb + off_tab + 8 * sizeof(float));
    a.s.phE = reinterpret_cast<const double2*>(sb + off_tab + 16 * sizeof(float));
    a.s.phH = reinterpret_cast<const double2*>(sb + off_tab + 16 * sizeof(float) + 8 * sizeof(double2));
    a.s.dft = reinterpret_cast<double2*>(sb + off_dft);
    a.s.n_tab = 8;                 // the zeroed source tables hold 8 steps
    a.s.n_coef = n_labels;
    a.ez_in = in[0]; a.hx_in = in[1]; a.hy_in = in[2];
    a.psiE_in = in[3]; a.psiH_in = in[4];
    a.ez_out = out[0]; a.hx_out = out[1]; a.hy_out = out[2];
    a.psiE_out = out[3]; a.psiH_out = out[4];
    a.seg_y0 = reinterpret_cast<const int*>(sb + off_seg);
    a.n_strips = n_strips;
    a.n_tasks = n_strips * (nb - 1);
    a.w_int = w_int;
    if (!launch_blocked(a, K, shape, 0, st))
        return fail(err, err_len, FDTD_EINVAL, "no blocked kernel instance for this step count");
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        std::snprintf(msg, sizeof msg, "launch: %s", cudaGetErrorString(e));
        return fail(err, err_len, FDTD_ECUDA, msg);
    }
    return FDTD_OK;
}
