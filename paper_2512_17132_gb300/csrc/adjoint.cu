// Discrete adjoint of R and T: gradients with respect to the per-cell
// (eps_r, sigma) and the per-label (n, kappa).
//
// fdtd_forward_checkpointed runs the forward loop from step 0 and stores the
// full state every C steps on the device. fdtd_backward then walks the
// segments last to first: it recomputes the segment from its checkpoint
// (the forward arithmetic exactly, so the same bits as the forward run) and
// stores on a device tape, for every step n, the two factors that the
// gradient sums take from the forward run: Ez^{n-1/2} and the factor of cb
// in the Ez update (curl^n with its CPML and TF/SF terms), 8 bytes per cell
// and step. It then applies, step by step in reverse, the transpose of every
// update of the leapfrog step:
//
//   forward step n                         reverse step n
//   Ez <- ca Ez + cb curl(H, psi_E)        k_adj_h: H monitor sources, transposes
//   Hx, Hy <- H + S dEz (+ psi_H)          of the H updates (psi_H carry), E
//   DFTs of Ez and averaged Hx             monitor source; k_adj_e: gca += lE
//                                          Ez^{n-1/2}, gcb += lE curl^n, transpose
//                                          of the E update (psi_E carry), ca lE
//
// Each reverse kernel recomputes the adjoint neighbour terms it needs
// instead of staging them, so the adjoint of Ez and the CPML carries are
// ping-ponged.
// Where rows split into float4s (nx % 4 == 0) the reverse kernels take four
// columns per thread (k_adj_h4, k_adj_e4); the scalar kernels serve the
// other widths; both give the same bits.
//
// in the library's units (Ez, eta0 H; ca, cb of Sec. 2.3). The monitor
// sources follow from J = wR R + wT T with R, T the Poynting ratios of
// Sec. 2.6 and the final DFT sums; the incident power does not depend on the
// cells. Per-segment FP32 gradient sums are added into FP64 totals, which
// are finally chained through ca(eps_r, sigma), cb(eps_r, sigma) and, for
// labelled handles, through eps_r = n^2 - k^2, sigma = 2 w0 eps0 n k
// (Sec. 2.2) with a per-label reduction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fdtd_internal.h"

using namespace fdtd;

namespace {

constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;

#define ACK(call)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);            \
            throw Fail{e_ == cudaErrorMemoryAllocation ? FDTD_ENOMEM : FDTD_ECUDA}; \
        }                                                                           \
    } while (0)

struct AdjArgs {
    int nx, ny, pitch, lpitch, P, js, jr, jt;
    float S;
    const uint8_t* labels;
    const float2* coef;
    const float2* cellcoef;
    const float* pml_e;
    const float* pml_h;
    const double2* phE;
    const double2* phH;
    const double2* dft;     // final DFT sums [4][nx]
    double kR, kT;          // dJ/d Re(E conj H) per monitor row
    float* lE;              // adjoint of Ez (the buffer the H reverse updates)
    float* lX; float* lY;
    float* gA; float* gB;   // FP32 per-segment sums
    const float* tE; const float* tC;   // tape of step n: Ez^{n-1/2}, factor of cb
    int n_coef;             // entries of coef (labelled handles)
    int64_t n_tab;          // table entries valid on the device (debug index checks)
    unsigned* dbg;          // error word of the debug index checks
};

__device__ __forceinline__ float2 cell_coef(const AdjArgs& a, int j, int i) {
    const size_t o = (size_t)j * a.pitch + i;
    return a.cellcoef ? a.cellcoef[o] : a.coef[a.labels[(size_t)j * a.lpitch + i]];
}

// monitor source of Hx^{n+1} at row j (rows jr, jr+1, jt, jt+1)
__device__ __forceinline__ float src_h(const AdjArgs& a, int j, int i, int64_t n) {
    double s = 0.0;
    const double2 ph = tab_n(a.phH, n, a.n_tab, a.dbg);
    if (j == a.jr || j == a.jr + 1) {
        const double2 e = a.dft[i];
        s += 0.5 * a.kR * (e.x * ph.x + e.y * ph.y);
    }
    if (j == a.jt || j == a.jt + 1) {
        const double2 e = a.dft[2 * a.nx + i];
        s += 0.5 * a.kT * (e.x * ph.x + e.y * ph.y);
    }
    return (float)s;
}

__device__ __forceinline__ float src_e(const AdjArgs& a, int j, int i, int64_t n) {
    double s = 0.0;
    const double2 pe = tab_n(a.phE, n, a.n_tab, a.dbg);
    if (j == a.jr) {
        const double2 hh = a.dft[a.nx + i];
        s += a.kR * (hh.x * pe.x + hh.y * pe.y);
    }
    if (j == a.jt) {
        const double2 hh = a.dft[3 * a.nx + i];
        s += a.kT * (hh.x * pe.x + hh.y * pe.y);
    }
    return (float)s;
}

// adjoint of d_ez at edge j (transpose of the Hx update, psi_H carry read
// from mH_in); x is the adjoint of Hx^{n+1} including its monitor source
__device__ __forceinline__ float adj_dez(const AdjArgs& a, int j, int i, int64_t n,
                                         const float* mH_in, float* mH_out) {
    if (j <= 0 || j >= a.ny) return 0.f;
    const size_t o = (size_t)j * a.pitch + i;
    float x = a.lX[o];
    if (j == a.jr || j == a.jr + 1 || j == a.jt || j == a.jt + 1) x = __fadd_rn(x, src_h(a, j, i, n));
    const int ph = pml_h_index(j, a.ny, a.P);
    if (ph >= 0) {
        const size_t q = (size_t)ph * a.pitch + i;
        const float sx = __fmul_rn(a.S, x);
        const float nu = __fadd_rn(sx, mH_in[q]);
        if (mH_out) mH_out[q] = __fmul_rn(a.pml_h[ph], nu);
        return __fmaf_rn(a.pml_h[2 * a.P + ph], nu, __fmul_rn(sx, a.pml_h[4 * a.P + ph]));
    }
    return __fmul_rn(a.S, x);
}

// Reverse of the H half-step: the adjoint of Ez^{n+1/2} collects the carried
// part, the transposes of both H updates and the E monitor source.
__global__ void k_adj_h(AdjArgs a, int64_t n, const float* __restrict__ mH_in,
                        float* __restrict__ mH_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= a.nx) return;
    const size_t o = (size_t)j * a.pitch + i;
    const int ir = (i + 1 == a.nx) ? 0 : i + 1;
    const float d0 = adj_dez(a, j, i, n, mH_in, mH_out);
    const float d1 = adj_dez(a, j + 1, i, n, mH_in, nullptr);
    float e = a.lE[o];
    e = __fadd_rn(e, __fmul_rn(a.S, __fsub_rn(a.lY[o], a.lY[(size_t)j * a.pitch + ir])));
    e = __fadd_rn(e, __fsub_rn(d0, d1));
    if (j == a.jr || j == a.jt) e = __fadd_rn(e, src_e(a, j, i, n));
    a.lE[o] = e;
}

// adjoint of curl (cbar) and of d_hx (psi_E carry from mE_in) at cell (j, i)
__device__ __forceinline__ void adj_curl(const AdjArgs& a, int j, int i, const float* lE_in,
                                         const float* mE_in, float* mE_out, float* cbar,
                                         float* ghx) {
    const size_t o = (size_t)j * a.pitch + i;
    const float2 c = cell_coef(a, j, i);
    const float cb = __fmul_rn(c.y, lE_in[o]);
    *cbar = cb;
    const int pe = pml_e_index(j, a.ny, a.P);
    if (pe >= 0) {
        const size_t q = (size_t)pe * a.pitch + i;
        const float rho = __fadd_rn(cb, mE_in[q]);
        if (mE_out) mE_out[q] = __fmul_rn(a.pml_e[pe], rho);
        *ghx = __fmaf_rn(a.pml_e[2 * a.P + pe], rho, __fmul_rn(cb, a.pml_e[4 * a.P + pe]));
    } else {
        *ghx = cb;
    }
}

// Reverse of the E half-step: gradient sums, transposes of d_hy and d_hx
// into the H adjoints (with the H monitor source made persistent) and
// lE <- ca lE into the other adjoint buffer.
__global__ void k_adj_e(AdjArgs a, int64_t n, const float* __restrict__ lE_in,
                        float* __restrict__ lE_out, const float* __restrict__ mE_in,
                        float* __restrict__ mE_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= a.nx) return;
    const size_t o = (size_t)j * a.pitch + i;
    const int il = (i == 0) ? a.nx - 1 : i - 1;
    const float eb = lE_in[o];
    // gradient sums with the taped factors of step n
    a.gA[o] = __fmaf_rn(eb, a.tE[o], a.gA[o]);
    a.gB[o] = __fmaf_rn(eb, a.tC[o], a.gB[o]);
    float c0, g0, cl, gu = 0.f, dummy;
    adj_curl(a, j, i, lE_in, mE_in, mE_out, &c0, &g0);
    adj_curl(a, j, il, lE_in, mE_in, nullptr, &cl, &dummy);
    if (j > 0) adj_curl(a, j - 1, i, lE_in, mE_in, nullptr, &dummy, &gu);
    a.lY[o] = __fadd_rn(a.lY[o], __fsub_rn(cl, c0));
    float x = a.lX[o];
    if (j == a.jr || j == a.jr + 1 || j == a.jt || j == a.jt + 1) x = __fadd_rn(x, src_h(a, j, i, n));
    a.lX[o] = __fadd_rn(x, __fsub_rn(gu, g0));
    lE_out[o] = __fmul_rn(cell_coef(a, j, i).x, eb);
}

// ---------------------------------------------------------------------------
// Four columns per thread (nx % 4 == 0): the same per-cell expressions as
// k_adj_h / k_adj_e, in the same order (bit-identical results), with float4
// loads and stores and the label coefficients in shared memory, so that each
// thread keeps four times the bytes in flight per load (the scalar kernels
// are latency-bound on chains of dependent loads).

__device__ __forceinline__ void ld4v(const float* p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void st4v(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// coefficients (ca, cb) of cells (j, i0..i0+3)
__device__ __forceinline__ void coef4(const AdjArgs& a, const float2* s_coef, int j, int i0,
                                      float2 (&c)[4]) {
    if (a.cellcoef) {
        const float4* p = reinterpret_cast<const float4*>(a.cellcoef + (size_t)j * a.pitch + i0);
        const float4 u = p[0], w = p[1];
        c[0] = make_float2(u.x, u.y); c[1] = make_float2(u.z, u.w);
        c[2] = make_float2(w.x, w.y); c[3] = make_float2(w.z, w.w);
    } else {
        const uint32_t L = *reinterpret_cast<const uint32_t*>(a.labels + (size_t)j * a.lpitch + i0);
#pragma unroll
        for (int q = 0; q < 4; ++q) c[q] = s_coef[(L >> (8 * q)) & 0xffu];
    }
}

__device__ __forceinline__ float2 coef1(const AdjArgs& a, const float2* s_coef, int j, int i) {
    const size_t o = (size_t)j * a.pitch + i;
    return a.cellcoef ? a.cellcoef[o] : s_coef[a.labels[(size_t)j * a.lpitch + i]];
}

__device__ __forceinline__ void load_coef_table(const AdjArgs& a, float2* s_coef) {
    if (!a.cellcoef)
        for (int t = threadIdx.x; t < a.n_coef; t += blockDim.x) s_coef[t] = a.coef[t];
    __syncthreads();
}

// adj_dez for columns i0..i0+3 of row j (mH_out row j written when given)
__device__ __forceinline__ void adj_dez4(const AdjArgs& a, int j, int i0, int64_t n,
                                         const float* mH_in, float* mH_out, float (&d)[4]) {
    if (j <= 0 || j >= a.ny) {
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = 0.f;
        return;
    }
    const size_t o = (size_t)j * a.pitch + i0;
    float x[4];
    ld4v(a.lX + o, x);
    if (j == a.jr || j == a.jr + 1 || j == a.jt || j == a.jt + 1)
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = __fadd_rn(x[q], src_h(a, j, i0 + q, n));
    const int ph = pml_h_index(j, a.ny, a.P);
    if (ph >= 0) {
        const size_t qq = (size_t)ph * a.pitch + i0;
        const float b = a.pml_h[ph], c = a.pml_h[2 * a.P + ph], ik = a.pml_h[4 * a.P + ph];
        float m[4], mo[4];
        ld4v(mH_in + qq, m);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float sx = __fmul_rn(a.S, x[q]);
            const float nu = __fadd_rn(sx, m[q]);
            mo[q] = __fmul_rn(b, nu);
            d[q] = __fmaf_rn(c, nu, __fmul_rn(sx, ik));
        }
        if (mH_out) st4v(mH_out + qq, mo);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = __fmul_rn(a.S, x[q]);
    }
}

__global__ void __launch_bounds__(256) k_adj_h4(AdjArgs a, int64_t n, const float* __restrict__ mH_in,
                                                float* __restrict__ mH_out) {
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y;
    if (i0 >= a.nx) return;
    const size_t o = (size_t)j * a.pitch + i0;
    float d0[4], d1[4], e[4], y[5];
    adj_dez4(a, j, i0, n, mH_in, mH_out, d0);
    adj_dez4(a, j + 1, i0, n, mH_in, nullptr, d1);
    ld4v(a.lE + o, e);
    ld4v(a.lY + o, *reinterpret_cast<float (*)[4]>(y));
    y[4] = a.lY[(size_t)j * a.pitch + ((i0 + 4 == a.nx) ? 0 : i0 + 4)];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        e[q] = __fadd_rn(e[q], __fmul_rn(a.S, __fsub_rn(y[q], y[q + 1])));
        e[q] = __fadd_rn(e[q], __fsub_rn(d0[q], d1[q]));
        if (j == a.jr || j == a.jt) e[q] = __fadd_rn(e[q], src_e(a, j, i0 + q, n));
    }
    st4v(a.lE + o, e);
}

// cbar and ghx (adj_curl) of cells (j, i0..i0+3); mE_out row j written when given
__device__ __forceinline__ void adj_curl4(const AdjArgs& a, const float2* s_coef, int j, int i0,
                                          const float* lE_in, const float* mE_in, float* mE_out,
                                          float (&cbar)[4], float (&ghx)[4]) {
    float2 c[4];
    coef4(a, s_coef, j, i0, c);
    float eb[4];
    ld4v(lE_in + (size_t)j * a.pitch + i0, eb);
#pragma unroll
    for (int q = 0; q < 4; ++q) cbar[q] = __fmul_rn(c[q].y, eb[q]);
    const int pe = pml_e_index(j, a.ny, a.P);
    if (pe >= 0) {
        const size_t qq = (size_t)pe * a.pitch + i0;
        const float b = a.pml_e[pe], cc = a.pml_e[2 * a.P + pe], ik = a.pml_e[4 * a.P + pe];
        float m[4], mo[4];
        ld4v(mE_in + qq, m);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float rho = __fadd_rn(cbar[q], m[q]);
            mo[q] = __fmul_rn(b, rho);
            ghx[q] = __fmaf_rn(cc, rho, __fmul_rn(cbar[q], ik));
        }
        if (mE_out) st4v(mE_out + qq, mo);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) ghx[q] = cbar[q];
    }
}

__global__ void __launch_bounds__(256) k_adj_e4(AdjArgs a, int64_t n, const float* __restrict__ lE_in,
                                                float* __restrict__ lE_out,
                                                const float* __restrict__ mE_in,
                                                float* __restrict__ mE_out) {
    __shared__ float2 s_coef[256];
    load_coef_table(a, s_coef);
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y;
    if (i0 >= a.nx) return;
    const size_t o = (size_t)j * a.pitch + i0;
    const int il = (i0 == 0) ? a.nx - 1 : i0 - 1;
    float eb[4];
    ld4v(lE_in + o, eb);
    // the taped factors of step n
    float te[4], curl[4];
    ld4v(a.tE + o, te);
    ld4v(a.tC + o, curl);
    float gA[4], gB[4];
    ld4v(a.gA + o, gA);
    ld4v(a.gB + o, gB);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        gA[q] = __fmaf_rn(eb[q], te[q], gA[q]);
        gB[q] = __fmaf_rn(eb[q], curl[q], gB[q]);
    }
    st4v(a.gA + o, gA);
    st4v(a.gB + o, gB);
    float c0[4], g0[4], gu[4];
    adj_curl4(a, s_coef, j, i0, lE_in, mE_in, mE_out, c0, g0);
    const float cl0 = __fmul_rn(coef1(a, s_coef, j, il).y, lE_in[(size_t)j * a.pitch + il]);
    if (j > 0) {
        float dummy[4];
        adj_curl4(a, s_coef, j - 1, i0, lE_in, mE_in, nullptr, dummy, gu);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) gu[q] = 0.f;
    }
    float ly[4], lx[4], leo[4];
    ld4v(a.lY + o, ly);
    ld4v(a.lX + o, lx);
    const bool mon = (j == a.jr || j == a.jr + 1 || j == a.jt || j == a.jt + 1);
    float2 cc[4];
    coef4(a, s_coef, j, i0, cc);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float cl = q ? c0[q - 1] : cl0;
        ly[q] = __fadd_rn(ly[q], __fsub_rn(cl, c0[q]));
        float x = lx[q];
        if (mon) x = __fadd_rn(x, src_h(a, j, i0 + q, n));
        lx[q] = __fadd_rn(x, __fsub_rn(gu[q], g0[q]));
        leo[q] = __fmul_rn(cc[q].x, eb[q]);
    }
    st4v(a.lY + o, ly);
    st4v(a.lX + o, lx);
    st4v(lE_out + o, leo);
}

__global__ void k_adj_flush(float* gA, float* gB, double* GA, double* GB, int nx, int ny,
                            int pitch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= nx) return;
    const size_t o = (size_t)j * pitch + i;
    GA[o] += (double)gA[o];
    GB[o] += (double)gB[o];
    gA[o] = 0.f;
    gB[o] = 0.f;
}

struct ChainArgs {
    int nx, ny, pitch, lpitch, n_labels;
    double S, dt, eps0, w;
    const uint8_t* labels;
    const double* mat;        // [n_labels][2] (n, k) for labelled handles
    const double* cell_eps;   // per-cell maps or null
    const double* cell_sig;
    const double* GA; const double* GB;
    double* g_eps; double* g_sig;   // dense ny*nx (device)
    double* g_lab;                  // [n_labels][2] or null
};

// dJ/d(eps_r), dJ/d(sigma) per cell and the per-label (n, kappa) sums
__global__ void k_adj_chain(ChainArgs a) {
    __shared__ double s_lab[256 * 2];
    for (int t = threadIdx.x; t < 512; t += blockDim.x) s_lab[t] = 0.0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < a.nx) {
        const size_t o = (size_t)j * a.pitch + i;
        double eps, sig, n = 0, k = 0;
        int l = 0;
        if (a.cell_eps) {
            eps = a.cell_eps[(size_t)j * a.nx + i];
            sig = a.cell_sig[(size_t)j * a.nx + i];
        } else {
            l = a.labels[(size_t)j * a.lpitch + i];
            n = a.mat[2 * l];
            k = a.mat[2 * l + 1];
            eps = n * n - k * k;
            sig = 2.0 * a.w * a.eps0 * n * k;
        }
        const double b = sig * a.dt / (2.0 * a.eps0 * eps);
        const double q = (1.0 + b) * (1.0 + b);
        const double dca_de = 2.0 * b / (eps * q);
        const double dca_ds = -a.dt / (a.eps0 * eps * q);
        const double dcb_de = -a.S / (eps * eps * q);
        const double dcb_ds = -a.S * a.dt / (2.0 * a.eps0 * eps * eps * q);
        const double ge = a.GA[o] * dca_de + a.GB[o] * dcb_de;
        const double gs = a.GA[o] * dca_ds + a.GB[o] * dcb_ds;
        a.g_eps[(size_t)j * a.nx + i] = ge;
        a.g_sig[(size_t)j * a.nx + i] = gs;
        if (a.g_lab) {
            atomicAdd(&s_lab[2 * l], ge * 2.0 * n + gs * 2.0 * a.w * a.eps0 * k);
            atomicAdd(&s_lab[2 * l + 1], -ge * 2.0 * k + gs * 2.0 * a.w * a.eps0 * n);
        }
    }
    __syncthreads();
    if (a.g_lab)
        for (int t = threadIdx.x; t < 2 * a.n_labels; t += blockDim.x)
            if (s_lab[t] != 0.0) atomicAdd(&a.g_lab[t], s_lab[t]);
}

// ---------------------------------------------------------------------------
// Temporally blocked reverse steps (labelled handles, nx % 4 == 0): K reverse
// steps n_top, n_top - 1, ..., n_top - K + 1 in one launch. The reverse step
// has the one-row reach of the forward step in both directions (the
// transpose of the H update looks one row down, that of the E update one row
// up), so the forward kernel's pipeline carries over: a warp owns a strip of
// 128 columns and a segment of rows, streams down the rows once, and level k
// (reverse step n_top - k) produces its output row r = t - k - 1 at
// iteration t from its input rows r and r + 1. Only level 0's input (the
// adjoint state lE, lX, lY) is read from memory and only level K's output
// written; the adjoint CPML carries travel between levels in a per-warp
// shared-memory ring; every level reads the taped gradient factors of its
// step for its output row r. Each cell's gradient sums are read, updated and written by
// the one lane that owns it, level after level, so they accumulate in the
// same order as with one reverse step per launch. Every expression is that
// of k_adj_h4 / k_adj_e4, so the gradients are bit for bit the same.
struct AdjBlockArgs {
    AdjArgs a;                          // lE, lX, lY, tE.. unused here
    const float* lE_in; const float* lX_in; const float* lY_in;
    float* lE_out; float* lX_out; float* lY_out;
    const float* mE_in; const float* mH_in;
    float* mE_out; float* mH_out;
    float* const* tape;                 // tape step base pointers; level k uses tape[m_top - k]
    int m_top;
    size_t tape_f;                      // floats per plane of a tape step (pitch * ny)
    const int* seg_y0;
    int n_strips, n_tasks, w_int;
};

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void ld4g(const float* p, float (&v)[4]) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void st4g(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Per-level pipeline registers: the level's pending input row r (lE, lX,
// lY and its label word), adj_dez of row r and g0 (the E-transpose term) of
// row r - 1.
template <int K>
struct AdjPipe {
    float E[K][4], X[K][4], Y[K][4], D[K][4], G[K][4];
    float GA[K][4], GB[K][4];           // running gradient sums of the pending row
    uint32_t L[K];
};

struct AdjLane {
    int gx, y0, y1, nx, ny, P;
    bool own;
};

// One level of one iteration: reverse step n = n_top - k turns the level's
// input rows r = q - 1 (pending) and q (iE, iX, iY, iL) into its output row
// r, returned in iE, iX, iY, iL as the input row of level k + 1. GENERAL is
// the path for iterations that touch a CPML, source, monitor or boundary
// row; both paths round identically.
template <int K, bool GENERAL>
__device__ __forceinline__ void adj_level(const AdjBlockArgs& b, const float2* s_coef,
                                          AdjPipe<K>& p, const int k, const int t,
                                          const int64_t n_top, const float4* tslot,
                                          float (&iE)[4], float (&iX)[4],
                                          float (&iY)[4], float (&iA)[4], float (&iB)[4],
                                          uint32_t& iL, const AdjLane& ln, float4* ringE,
                                          float4* ringH) {
    const AdjArgs& a = b.a;
    const int q = t - k, r = q - 1;
    const int64_t n = n_top - k;
    const float S = a.S;
    const size_t pitch = (size_t)a.pitch;
    const bool r_ok = !GENERAL || (r >= 0 && r < ln.ny);
    // 1. transpose of the Hx update at edge q (adj_dez), psi_H carry of row q
    float dq[4];
    if (!GENERAL) {
#pragma unroll
        for (int c = 0; c < 4; ++c) dq[c] = __fmul_rn(S, iX[c]);
    } else if (q <= 0 || q >= ln.ny) {
#pragma unroll
        for (int c = 0; c < 4; ++c) dq[c] = 0.f;
    } else {
        float x[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = iX[c];
        if (q == a.jr || q == a.jr + 1 || q == a.jt || q == a.jt + 1)
#pragma unroll
            for (int c = 0; c < 4; ++c) x[c] = __fadd_rn(x[c], src_h(a, q, ln.gx + c, n));
        const int ph = pml_h_index(q, ln.ny, ln.P);
        if (ph >= 0 && index_ok(ph < 2 * ln.P, kSitePsiRow, a.dbg)) {
            const float bb = a.pml_h[ph], cc = a.pml_h[2 * a.P + ph], ik = a.pml_h[4 * a.P + ph];
            float m[4], mo[4];
            if (k == 0) {
                ld4g(b.mH_in + (size_t)ph * pitch + ln.gx, m);
            } else {
                const float4 v = ringH[(q % K) * 32];
                m[0] = v.x; m[1] = v.y; m[2] = v.z; m[3] = v.w;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float sx = __fmul_rn(S, x[c]);
                const float nu = __fadd_rn(sx, m[c]);
                mo[c] = __fmul_rn(bb, nu);
                dq[c] = __fmaf_rn(cc, nu, __fmul_rn(sx, ik));
            }
            if (k == K - 1) {
                if (ln.own && q >= ln.y0 && q < ln.y1) st4g(b.mH_out + (size_t)ph * pitch + ln.gx, mo);
            } else {
                ringH[(q % K) * 32] = make_float4(mo[0], mo[1], mo[2], mo[3]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) dq[c] = __fmul_rn(S, x[c]);
        }
    }
    float oE[4], oX[4], oY[4], g0[4], oA[4], oB[4];
    if (r_ok) {
        // 2. the adjoint of Ez^{n+1/2} after the H transposes (k_adj_h)
        const float yR = __shfl_down_sync(kFull, p.Y[k][0], 1);
        float eh[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            eh[c] = __fadd_rn(p.E[k][c], __fmul_rn(S, __fsub_rn(p.Y[k][c], c < 3 ? p.Y[k][c + 1] : yR)));
            eh[c] = __fadd_rn(eh[c], __fsub_rn(p.D[k][c], dq[c]));
        }
        if (GENERAL && (r == a.jr || r == a.jt))
#pragma unroll
            for (int c = 0; c < 4; ++c) eh[c] = __fadd_rn(eh[c], src_e(a, r, ln.gx + c, n));
        // 3. gradient sums with the taped factors of step n, row r (staged in
        // shared memory one iteration ahead); the sums travel with the row
        // from level to level (read by level 0, written after level K - 1),
        // level order = step order
        const float4 te = tslot[0], tc = tslot[32];
        const float tE[4] = {te.x, te.y, te.z, te.w}, curl[4] = {tc.x, tc.y, tc.z, tc.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            oA[c] = __fmaf_rn(eh[c], tE[c], p.GA[k][c]);
            oB[c] = __fmaf_rn(eh[c], curl[c], p.GB[k][c]);
        }
        const int pe = GENERAL ? pml_e_index(r, ln.ny, ln.P) : -1;
        // 4. transpose of the Ez update (adj_curl of row r), psi_E carry of row r
        const uint32_t L = p.L[k];
        float2 cf[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) cf[c] = s_coef[(L >> (8 * c)) & 0xffu];
        float cbar[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) cbar[c] = __fmul_rn(cf[c].y, eh[c]);
        if (GENERAL && pe >= 0 && index_ok(pe < 2 * ln.P, kSitePsiRow, a.dbg)) {
            const float bb = a.pml_e[pe], cc = a.pml_e[2 * a.P + pe], ik = a.pml_e[4 * a.P + pe];
            float m[4], mo[4];
            if (k == 0) {
                ld4g(b.mE_in + (size_t)pe * pitch + ln.gx, m);
            } else {
                const float4 v = ringE[(r % K) * 32];
                m[0] = v.x; m[1] = v.y; m[2] = v.z; m[3] = v.w;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float rho = __fadd_rn(cbar[c], m[c]);
                mo[c] = __fmul_rn(bb, rho);
                g0[c] = __fmaf_rn(cc, rho, __fmul_rn(cbar[c], ik));
            }
            if (k == K - 1) {
                if (ln.own && r >= ln.y0 && r < ln.y1) st4g(b.mE_out + (size_t)pe * pitch + ln.gx, mo);
            } else {
                ringE[(r % K) * 32] = make_float4(mo[0], mo[1], mo[2], mo[3]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) g0[c] = cbar[c];
        }
        const float cl0 = __shfl_up_sync(kFull, cbar[3], 1);
        const bool mon = GENERAL && (r == a.jr || r == a.jr + 1 || r == a.jt || r == a.jt + 1);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float cl = c ? cbar[c - 1] : cl0;
            const float gu = (GENERAL && r == 0) ? 0.f : p.G[k][c];
            oY[c] = __fadd_rn(p.Y[k][c], __fsub_rn(cl, cbar[c]));
            float x = p.X[k][c];
            if (mon) x = __fadd_rn(x, src_h(a, r, ln.gx + c, n));
            oX[c] = __fadd_rn(x, __fsub_rn(gu, g0[c]));
            oE[c] = __fmul_rn(cf[c].x, eh[c]);
        }
    } else {
        // outside the grid (warp-uniform): a zero row, which reaches no stored row
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            oE[c] = 0.f; oX[c] = 0.f; oY[c] = 0.f; g0[c] = 0.f; oA[c] = 0.f; oB[c] = 0.f;
        }
    }
    // the input row q becomes the level's pending row; row r moves up a level
    const uint32_t oL = p.L[k];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        p.E[k][c] = iE[c]; p.X[k][c] = iX[c]; p.Y[k][c] = iY[c];
        p.D[k][c] = dq[c]; p.G[k][c] = g0[c];
        p.GA[k][c] = iA[c]; p.GB[k][c] = iB[c];
        iE[c] = oE[c]; iX[c] = oX[c]; iY[c] = oY[c]; iA[c] = oA[c]; iB[c] = oB[c];
    }
    p.L[k] = iL;
    iL = oL;
}

constexpr int kAdjRing = 2;   // ring slots of the blocked reverse kernel's staged rows (3 measured slower)

__device__ __forceinline__ void cp16(void* smem, const void* gmem, int bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes)
                 : "memory");
}

template <int K>
__global__ void __launch_bounds__(32) k_adj_blocked(const AdjBlockArgs b, const int64_t n_top) {
    __shared__ float2 s_coef[256];
    __shared__ float4 s_ring[2][K][32];
    // tape rows of each level, kAdjRing iterations in flight:
    // [slot][level][Ez^{n-1/2}, factor of cb][lane]
    __shared__ float4 s_tape[kAdjRing][K][2][32];
    // level-0 input row (lE, lX, lY, gA, gB) and its labels, same slots
    __shared__ float4 s_in[kAdjRing][5][32];
    __shared__ uint32_t s_lab[kAdjRing][32];
    for (int i = threadIdx.x; i < b.a.n_coef; i += 32) s_coef[i] = b.a.coef[i];
    __syncwarp();
    if ((int)blockIdx.x >= b.n_tasks) return;
    const AdjArgs& a = b.a;
    constexpr int H = ((K + 3) / 4) * 4;
    const int lane = threadIdx.x & 31;
    const int strip = blockIdx.x % b.n_strips;
    const int seg = blockIdx.x / b.n_strips;
    AdjLane ln;
    ln.y0 = b.seg_y0[seg];
    ln.y1 = b.seg_y0[seg + 1];
    ln.nx = a.nx; ln.ny = a.ny; ln.P = a.P;
    const int xl = 4 * lane;
    const int xg_pre = strip * b.w_int - H + xl;
    ln.gx = ((xg_pre % ln.nx) + ln.nx) % ln.nx;
    const bool col_ok = index_ok(ln.gx >= 0 && ln.gx + 4 <= ln.nx, kSiteRingColumn, a.dbg);
    ln.own = (xl >= H) && (xl < H + b.w_int) && (xg_pre < ln.nx) && col_ok;
    float4* ringE = &s_ring[0][0][lane];
    float4* ringH = &s_ring[1][0][lane];
    const float* tbs[K];                 // tape step of each level
#pragma unroll
    for (int k = 0; k < K; ++k) tbs[k] = b.tape[b.m_top - k];
    AdjPipe<K> p;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            p.E[k][c] = 0.f; p.X[k][c] = 0.f; p.Y[k][c] = 0.f;
            p.D[k][c] = 0.f; p.G[k][c] = 0.f;
            p.GA[k][c] = 0.f; p.GB[k][c] = 0.f;
        }
        p.L[k] = 0u;
    }
    const size_t pitch = (size_t)a.pitch, lpitch = (size_t)a.lpitch;
    const int ny = ln.ny, P = ln.P;
    const int t_begin = (ln.y0 == 0) ? 0 : (ln.y0 - K);
    const int t_end = ln.y1 + K;
    const int lo = max(P, 1) + K;
    const int sp[5] = {a.js, a.jr, a.jr + 1, a.jt, a.jt + 1};
    auto is_lean = [&](int t) {
        bool f = (t >= lo) && (t < ny - P);
#pragma unroll
        for (int s = 0; s < 5; ++s) f = f && ((unsigned)(t - sp[s]) > (unsigned)K);
        return f;
    };
    // tape rows needed at iteration t: level k reads both factors of row
    // t - k - 1 of its step; rows outside the grid are zero-filled
    float4* tape_lane = &s_tape[0][0][0][lane];
    auto stage_tape = [&](int t) {
        const int slot = t % kAdjRing;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int r = t - k - 1;
            const bool rok = r >= 0 && r < ny && col_ok;
            const float* tb = tbs[k];
            const size_t orow = (size_t)(rok ? r : 0) * pitch + ln.gx;
            float4* dst = tape_lane + (slot * K + k) * 64;
            cp16(dst, tb + orow, rok ? 16 : 0);
            cp16(dst + 32, tb + b.tape_f + orow, rok ? 16 : 0);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    // level-0 input rows (adjoint state and gradient sums) and labels, staged
    // with the tape rows of the same iteration (zero outside the grid)
    auto stage_in = [&](int row) {
        const int slot = row % kAdjRing;
        const bool ok = row >= 0 && row < ny && col_ok;
        const size_t o = (size_t)(ok ? row : 0) * pitch + ln.gx;
        const int nb = ok ? 16 : 0;
        float4* d = &s_in[0][0][lane] + slot * 160;
        cp16(d, b.lE_in + o, nb);
        cp16(d + 32, b.lX_in + o, nb);
        cp16(d + 64, b.lY_in + o, nb);
        cp16(d + 96, a.gA + o, nb);
        cp16(d + 128, a.gB + o, nb);
        const unsigned sa = (unsigned)__cvta_generic_to_shared(&s_lab[slot][lane]);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa),
                     "l"(a.labels + (size_t)(ok ? row : 0) * lpitch + ln.gx), "r"(ok ? 4 : 0)
                     : "memory");
    };
    // one commit group per iteration, kAdjRing - 1 iterations ahead
#pragma unroll
    for (int d = 0; d < kAdjRing - 1; ++d) {
        stage_in(t_begin + d);
        stage_tape(t_begin + d);
    }
#pragma unroll 1
    for (int t = t_begin; t < t_end; ++t) {
        stage_in(t + kAdjRing - 1);
        stage_tape(t + kAdjRing - 1);
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kAdjRing - 1) : "memory");  // iteration t
        float iE[4], iX[4], iY[4], iA[4], iB[4];
        {
            const float4* src = &s_in[0][0][lane] + (t % kAdjRing) * 160;
            float* dst[5] = {iE, iX, iY, iA, iB};
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                const float4 v = src[32 * f];
                dst[f][0] = v.x; dst[f][1] = v.y; dst[f][2] = v.z; dst[f][3] = v.w;
            }
        }
        uint32_t iL = s_lab[t % kAdjRing][lane];
        const float4* ts = tape_lane + (t % kAdjRing) * K * 64;
        if (is_lean(t)) {
#pragma unroll
            for (int k = 0; k < K; ++k)
                adj_level<K, false>(b, s_coef, p, k, t, n_top, ts + k * 64, iE, iX, iY, iA, iB,
                                    iL, ln, ringE, ringH);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k)
                adj_level<K, true>(b, s_coef, p, k, t, n_top, ts + k * 64, iE, iX, iY, iA, iB,
                                   iL, ln, ringE, ringH);
        }
        const int ro = t - K;
        if (ln.own && ro >= ln.y0 && ro < ln.y1) {
            const size_t o = (size_t)ro * pitch + ln.gx;
            st4g(b.lE_out + o, iE);
            st4g(b.lX_out + o, iX);
            st4g(b.lY_out + o, iY);
            st4g(a.gA + o, iA);
            st4g(a.gB + o, iB);
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

int adj_blocked_per_sm(int K) {
    int v = 0;
    cudaError_t e = cudaSuccess;
    switch (K) {
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_adj_blocked<1>, 32, 0); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_adj_blocked<2>, 32, 0); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_adj_blocked<3>, 32, 0); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_adj_blocked<4>, 32, 0); break;
        default: return 0;
    }
    return e == cudaSuccess ? v : 0;
}

// Segment plan of the blocked reverse kernel for depth K: the forward
// planner's cuts (segment_bounds) for the segment count that minimises
// waves x (rows + 2K) with this kernel's own occupancy and general-path
// weight.
struct AdjPlan {
    int K = 0, n_strips = 0, n_segs = 0, w_int = 0;
    int* d_seg = nullptr;
};

AdjPlan make_adj_plan(fdtd_handle* h, int K) {
    AdjPlan pl;
    pl.K = K;
    const int halo = (K + 3) / 4 * 4;
    pl.w_int = 128 - 2 * halo;
    pl.n_strips = (h->g.nx + pl.w_int - 1) / pl.w_int;
    int per_sm = adj_blocked_per_sm(K);
    if (per_sm <= 0) per_sm = 8;
    const int64_t W = (int64_t)sm_count(h) * per_sm;
    const int ny = h->g.ny;
    double best = 1e300;
    int seg = ny;
    for (int n = 1; n <= std::max(1, ny / (K + 1)); ++n) {
        const int64_t waves = ((int64_t)n * pl.n_strips + W - 1) / W;
        const double rows = std::ceil((double)ny / n);
        const double cost = (double)waves * (rows + 2.0 * K);
        if (cost < best - 1e-9) { best = cost; seg = (int)rows; }
    }
    const double wg = h->opt_weight > 0.0 ? h->opt_weight : kReverseGeneralCost;
    const std::vector<int> bnd = segment_bounds(h->g, std::max(seg, K + 1), K, 0, wg);
    pl.n_segs = (int)bnd.size() - 1;
    ACK(cudaMalloc(&pl.d_seg, bnd.size() * sizeof(int)));
    ACK(cudaMemcpy(pl.d_seg, bnd.data(), bnd.size() * sizeof(int), cudaMemcpyHostToDevice));
    return pl;
}

bool launch_adj_blocked(const AdjBlockArgs& b, int K, int64_t n_top, cudaStream_t st) {
    const unsigned grid = (unsigned)b.n_tasks;
    switch (K) {
        case 1: k_adj_blocked<1><<<grid, 32, 0, st>>>(b, n_top); return true;
        case 2: k_adj_blocked<2><<<grid, 32, 0, st>>>(b, n_top); return true;
        case 3: k_adj_blocked<3><<<grid, 32, 0, st>>>(b, n_top); return true;
        case 4: k_adj_blocked<4><<<grid, 32, 0, st>>>(b, n_top); return true;
        default: return false;
    }
}

size_t state_floats(const fdtd_handle* h) {
    return (size_t)3 * h->pitch * h->g.ny + (size_t)2 * std::max(2 * h->g.pml_cells, 1) * h->pitch;
}

// views of one packed state: Ez, Hx, Hy, psi_E, psi_H
struct StateView {
    float *E, *X, *Y, *PE, *PH;
};
StateView view(const fdtd_handle* h, float* base) {
    const size_t f = (size_t)h->pitch * h->g.ny;
    const size_t p = (size_t)std::max(2 * h->g.pml_cells, 1) * h->pitch;
    return {base, base + f, base + 2 * f, base + 3 * f, base + 3 * f + p};
}

void copy_state_out(fdtd_handle* h, float* dst) {
    const size_t f = (size_t)h->pitch * h->g.ny * sizeof(float);
    const size_t p = (size_t)std::max(2 * h->g.pml_cells, 1) * h->pitch * sizeof(float);
    const StateView v = view(h, dst);
    const int c = h->cur;
    ACK(cudaMemcpyAsync(v.E, h->ez[c], f, cudaMemcpyDeviceToDevice, h->stream));
    ACK(cudaMemcpyAsync(v.X, h->hx[c], f, cudaMemcpyDeviceToDevice, h->stream));
    ACK(cudaMemcpyAsync(v.Y, h->hy[c], f, cudaMemcpyDeviceToDevice, h->stream));
    ACK(cudaMemcpyAsync(v.PE, h->psiE[c], p, cudaMemcpyDeviceToDevice, h->stream));
    ACK(cudaMemcpyAsync(v.PH, h->psiH[c], p, cudaMemcpyDeviceToDevice, h->stream));
}

// One forward step n from state `in` to state `out` (no monitor sums) with
// the per-step kernels, storing the step's gradient factors at `tape`
// (grids that the blocked kernel does not take: per-cell materials or
// nx % 4 != 0).
void step_to_tape(fdtd_handle* h, const StateView& in, const StateView& out, int64_t n,
                  float* tape, double2* dummy) {
    StepArgs s = step_args(h);
    s.dft = dummy;
    const size_t f = (size_t)h->pitch * h->g.ny * sizeof(float);
    const size_t p = (size_t)std::max(2 * h->g.pml_cells, 1) * h->pitch * sizeof(float);
    ACK(cudaMemcpyAsync(out.E, in.E, f, cudaMemcpyDeviceToDevice, h->stream));
    ACK(cudaMemcpyAsync(out.X, in.X, f, cudaMemcpyDeviceToDevice, h->stream));
    ACK(cudaMemcpyAsync(out.Y, in.Y, f, cudaMemcpyDeviceToDevice, h->stream));
    ACK(cudaMemcpyAsync(out.PE, in.PE, p, cudaMemcpyDeviceToDevice, h->stream));
    ACK(cudaMemcpyAsync(out.PH, in.PH, p, cudaMemcpyDeviceToDevice, h->stream));
    launch_naive_step(s, out.E, out.X, out.Y, out.PE, out.PH, n, h->stream, tape,
                      (size_t)h->pitch * h->g.ny);
}

// Recompute K steps n..n+K-1 from state `in` in one blocked launch (code
// shape 6, or 4 for more than 16 labels): the launch writes the final state
// to `out` and the gradient factors of step n+k to tape_ptrs[k] (device
// array of tape step base pointers); the same arithmetic as K one-step
// launches, so the same bits.
void steps_to_tape(fdtd_handle* h, const StateView& in, const StateView& out, int K, int64_t n,
                   float* const* tape_ptrs, double2* dummy) {
    StepArgs s = step_args(h);
    s.dft = dummy;
    // code shape 6 (label-pair table, paired lean path) where the labels fit
    const int shape = pair_shape_ok(false, h->maps, h->n_labels) ? 6 : 4;
    const int keep = h->opt_seg;
    h->opt_seg = 0;
    BlockPlan& pl = plan_for(h, h->tape_plans, K, shape,
                             h->opt_weight > 0.0 ? h->opt_weight : kTapeGeneralCost);
    h->opt_seg = keep;
    BlockedArgs b{};
    b.s = s;
    b.ez_in = in.E; b.hx_in = in.X; b.hy_in = in.Y;
    b.ez_out = out.E; b.hx_out = out.X; b.hy_out = out.Y;
    b.psiE_in = in.PE; b.psiH_in = in.PH; b.psiE_out = out.PE; b.psiH_out = out.PH;
    b.seg_y0 = pl.d_seg_y0;
    b.n_strips = pl.n_strips;
    b.n_tasks = pl.n_strips * pl.n_segs;
    b.w_int = pl.w_int;
    b.tape = tape_ptrs;
    b.tape_f = (size_t)h->pitch * h->g.ny;
    launch_blocked(b, K, shape, n, h->stream);
}

}  // namespace

extern "C" {

int fdtd_forward_checkpointed(fdtd_handle* h, int64_t steps, int32_t every) {
    if (!h) return FDTD_EINVAL;
    try {
        if (steps < 1 || every < 1) {
            h->err = "fdtd_forward_checkpointed: need steps >= 1 and every >= 1";
            return FDTD_EINVAL;
        }
        if (h->src.polarization != FDTD_POL_S) {
            h->err = "fdtd_forward_checkpointed: the adjoint covers S (TMz) handles only";
            return FDTD_EINVAL;
        }
        ACK(cudaSetDevice(h->device));
        const int rc = fdtd_reset(h);
        if (rc != FDTD_OK) return rc;
        const int64_t n_ck = (steps + every - 1) / every;
        const size_t sf = state_floats(h);
        if ((int64_t)h->ck.size() != n_ck || h->ck_floats != sf) {
            ACK(cudaStreamSynchronize(h->stream));
            for (auto& c : h->ck) { cudaFree(c); c = nullptr; }
            h->ck.assign((size_t)n_ck, nullptr);
            for (auto& c : h->ck) ACK(cudaMalloc(&c, sf * sizeof(float)));
            h->ck_floats = sf;
        }
        h->adj_valid = false;
        for (int64_t c = 0; c < n_ck; ++c) {
            copy_state_out(h, h->ck[(size_t)c]);
            const int r = fdtd_run(h, std::min<int64_t>(every, steps - c * every));
            if (r != FDTD_OK) return r;
        }
        h->adj_steps = steps;
        h->adj_every = every;
        h->adj_valid = true;
        return FDTD_OK;
    } catch (const Fail& f) {
        return f.code;
    }
}

int fdtd_backward(fdtd_handle* h, double wR, double wT, double* g_eps, double* g_sigma,
                  double* g_label, double out[3]) {
    if (!h) return FDTD_EINVAL;
    std::vector<AdjPlan> adj_plans;
    float* buf = nullptr;
    double* dbl = nullptr;
    double2* dummy = nullptr;
    auto cleanup = [&]() {
        for (auto& pl : adj_plans) if (pl.d_seg) cudaFree(pl.d_seg);
        if (buf) cudaFree(buf);
        if (dbl) cudaFree(dbl);
        if (dummy) cudaFree(dummy);
    };
    try {
        if (!h->adj_valid || h->n != h->adj_steps) {
            h->err = "fdtd_backward: run fdtd_forward_checkpointed first (and no steps since)";
            return FDTD_ESTATE;
        }
        ACK(cudaSetDevice(h->device));
        double flux[3];
        int rc = fdtd_flux_raw(h, flux);
        if (rc != FDTD_OK) return rc;
        double R = 0, T = 0;
        rc = fdtd_flux(h, &R, &T);
        if (rc != FDTD_OK) return rc;
        const double s0 = h->h_flux[2];
        if (!(s0 != 0.0)) {
            h->err = "fdtd_backward: no incident power at t_row (run longer)";
            return FDTD_ESTATE;
        }
        const fdtd_grid& g = h->g;
        const int nx = g.nx, ny = g.ny, pitch = h->pitch;
        const size_t f = (size_t)pitch * ny;
        const size_t pr = (size_t)std::max(2 * g.pml_cells, 1) * pitch;
        const int every = h->adj_every;
        const int64_t steps = h->adj_steps;
        // the tape: per step of a segment, Ez^{n-1/2} and the factor of cb
        // (f floats each); two state buffers carry the recompute; a device
        // array holds the tape steps' base pointers for the multi-step
        // recompute (labelled grids with nx % 4 == 0). The handle keeps them
        // for the next fdtd_backward of the same size.
        const size_t sf = state_floats(h);
        const size_t n_tape = (size_t)std::min<int64_t>(every, steps);
        if (h->adj_tape.size() != n_tape || h->adj_tape_floats != 2 * f) {
            ACK(cudaStreamSynchronize(h->stream));
            for (auto& t : h->adj_tape) cudaFree(t);
            for (float*& q : h->adj_state) { if (q) cudaFree(q); q = nullptr; }
            if (h->d_adj_tape_ptrs) cudaFree(h->d_adj_tape_ptrs);
            h->d_adj_tape_ptrs = nullptr;
            h->adj_tape.assign(n_tape, nullptr);
            h->adj_tape_floats = 0;
            for (auto& t : h->adj_tape) ACK(cudaMalloc(&t, 2 * f * sizeof(float)));
            for (float*& q : h->adj_state) ACK(cudaMalloc(&q, sf * sizeof(float)));
            ACK(cudaMalloc(&h->d_adj_tape_ptrs, n_tape * sizeof(float*)));
            ACK(cudaMemcpy(h->d_adj_tape_ptrs, h->adj_tape.data(), n_tape * sizeof(float*),
                           cudaMemcpyHostToDevice));
            h->adj_tape_floats = 2 * f;
        }
        const std::vector<float*>& tape = h->adj_tape;
        float* const* st = h->adj_state;
        float* const* d_tape_ptrs = h->d_adj_tape_ptrs;
        const bool multi = !h->maps && nx % 4 == 0;
        // lE[2] lX lY gA gB (f each) + mE[2] mH[2] (pr each) + the second lX, lY
        // buffers of the blocked reverse kernel (f each)
        ACK(cudaMalloc(&buf, (8 * f + 4 * pr) * sizeof(float)));
        ACK(cudaMemsetAsync(buf, 0, (8 * f + 4 * pr) * sizeof(float), h->stream));
        ACK(cudaMalloc(&dbl, 2 * f * sizeof(double)));
        ACK(cudaMemsetAsync(dbl, 0, 2 * f * sizeof(double), h->stream));
        ACK(cudaMalloc(&dummy, (size_t)4 * nx * sizeof(double2)));
        AdjArgs a{};
        a.nx = nx; a.ny = ny; a.pitch = pitch; a.lpitch = h->lpitch; a.P = g.pml_cells;
        a.js = g.tfsf_row; a.jr = g.r_row; a.jt = g.t_row; a.S = (float)h->S;
        a.labels = h->labels; a.coef = h->coef; a.cellcoef = h->cellcoef;
        a.pml_e = h->pml_e; a.pml_h = h->pml_h;
        a.phE = h->d_phE; a.phH = h->d_phH; a.dft = h->dft;
        a.kR = wR / (-(double)nx * s0);
        a.kT = wT / ((double)nx * s0);
        float* lEb[2] = {buf, buf + f};
        a.lX = buf + 2 * f; a.lY = buf + 3 * f; a.gA = buf + 4 * f; a.gB = buf + 5 * f;
        float* mEb[2] = {buf + 6 * f, buf + 6 * f + pr};
        float* mHb[2] = {buf + 6 * f + 2 * pr, buf + 6 * f + 3 * pr};
        float* lXb[2] = {buf + 2 * f, buf + 6 * f + 4 * pr};
        float* lYb[2] = {buf + 3 * f, buf + 7 * f + 4 * pr};
        int pe_cur = 0, ph_cur = 0, le_cur = 0, lxy_cur = 0;
        // reverse steps per launch: K-step blocked launches (labelled grids with
        // nx % 4 == 0), else one launch pair per step
        const int kb = (multi && h->opt_adj_block > 0) ? std::min(h->opt_adj_block, 4) : 0;
        double* GA = dbl;
        double* GB = dbl + f;
        const dim3 blk(256), grd((nx + 255) / 256, ny);
        // four columns per thread where rows split into float4s
        const bool vec4 = (nx % 4 == 0);
        const dim3 grd4((nx / 4 + 255) / 256, ny);
        a.n_coef = h->n_labels;
        a.n_tab = table_limit(h);
        a.dbg = h->d_dbg;
        const int64_t n_seg = (steps + every - 1) / every;
        for (int64_t c = n_seg - 1; c >= 0; --c) {
            const int64_t c0 = c * every;
            const int L = (int)std::min<int64_t>(every, steps - c0);
            // recompute steps c0 .. c0+L-1 from the checkpoint (read only)
            StateView in = view(h, h->ck[(size_t)c]);
            int so = 0;
            if (multi) {
                const int Kmax = std::min(std::max(h->opt_block, 1), blocked_max_K());
                for (int m = 0; m < L;) {
                    const int Kr = std::min(Kmax, L - m);
                    const StateView out = view(h, st[so]);
                    steps_to_tape(h, in, out, Kr, c0 + m, d_tape_ptrs + m, dummy);
                    h->total_launches += 1;
                    in = out;
                    so ^= 1;
                    m += Kr;
                }
            } else {
                for (int m = 0; m < L; ++m) {
                    const StateView out = view(h, st[so]);
                    step_to_tape(h, in, out, c0 + m, tape[m], dummy);
                    h->total_launches += 3;
                    in = out;
                    so ^= 1;
                }
            }
            for (int m_top = L - 1; kb > 0 && m_top >= 0;) {
                const int Kr = std::min(kb, m_top + 1);
                AdjPlan* plp = nullptr;
                for (auto& q : adj_plans)
                    if (q.K == Kr) plp = &q;
                if (!plp) {
                    adj_plans.push_back(make_adj_plan(h, Kr));
                    plp = &adj_plans.back();
                }
                const AdjPlan& pl = *plp;
                AdjBlockArgs bb{};
                bb.a = a;
                bb.lE_in = lEb[le_cur]; bb.lE_out = lEb[le_cur ^ 1];
                bb.lX_in = lXb[lxy_cur]; bb.lX_out = lXb[lxy_cur ^ 1];
                bb.lY_in = lYb[lxy_cur]; bb.lY_out = lYb[lxy_cur ^ 1];
                bb.mE_in = mEb[pe_cur]; bb.mE_out = mEb[pe_cur ^ 1];
                bb.mH_in = mHb[ph_cur]; bb.mH_out = mHb[ph_cur ^ 1];
                bb.tape = d_tape_ptrs;
                bb.m_top = m_top;
                bb.tape_f = f;
                bb.seg_y0 = pl.d_seg;
                bb.n_strips = pl.n_strips;
                bb.n_tasks = pl.n_strips * pl.n_segs;
                bb.w_int = pl.w_int;
                if (!launch_adj_blocked(bb, Kr, c0 + m_top, h->stream)) {
                    h->err = "fdtd_backward: no blocked reverse kernel for this depth";
                    throw Fail{FDTD_EINVAL};
                }
                le_cur ^= 1; lxy_cur ^= 1; pe_cur ^= 1; ph_cur ^= 1;
                h->total_launches += 1;
                m_top -= Kr;
            }
            for (int m = L - 1; kb == 0 && m >= 0; --m) {
                const int64_t n = c0 + m;
                a.tE = tape[m];
                a.tC = tape[m] + f;
                a.lE = lEb[le_cur];
                if (vec4) {
                    k_adj_h4<<<grd4, blk, 0, h->stream>>>(a, n, mHb[ph_cur], mHb[ph_cur ^ 1]);
                    ph_cur ^= 1;
                    k_adj_e4<<<grd4, blk, 0, h->stream>>>(a, n, lEb[le_cur], lEb[le_cur ^ 1],
                                                          mEb[pe_cur], mEb[pe_cur ^ 1]);
                } else {
                    k_adj_h<<<grd, blk, 0, h->stream>>>(a, n, mHb[ph_cur], mHb[ph_cur ^ 1]);
                    ph_cur ^= 1;
                    k_adj_e<<<grd, blk, 0, h->stream>>>(a, n, lEb[le_cur], lEb[le_cur ^ 1],
                                                        mEb[pe_cur], mEb[pe_cur ^ 1]);
                }
                pe_cur ^= 1;
                le_cur ^= 1;
            }
            k_adj_flush<<<grd, blk, 0, h->stream>>>(a.gA, a.gB, GA, GB, nx, ny, pitch);
            h->total_launches += (kb ? 0 : 2 * L) + 1;
            ACK(cudaGetLastError());
        }
        // chain rule to (eps_r, sigma) per cell and (n, kappa) per label
        double* d_ge = nullptr;
        double* d_gs = nullptr;
        double* d_gl = nullptr;
        double* d_mat = nullptr;
        const size_t cells = (size_t)nx * ny;
        ACK(cudaMalloc(&d_ge, cells * sizeof(double)));
        ACK(cudaMalloc(&d_gs, cells * sizeof(double)));
        ChainArgs ch{};
        ch.nx = nx; ch.ny = ny; ch.pitch = pitch; ch.lpitch = h->lpitch; ch.n_labels = h->n_labels;
        ch.S = h->S; ch.dt = g.dt;
        ch.eps0 = 1.0 / (4.0e-7 * kPi * kC0 * kC0);
        ch.w = 2.0 * kPi * kC0 / h->src.lambda0;
        ch.labels = h->labels;
        ch.GA = GA; ch.GB = GB; ch.g_eps = d_ge; ch.g_sig = d_gs;
        if (h->maps) {
            ch.cell_eps = h->cell_eps;
            ch.cell_sig = h->cell_sig;
        } else {
            std::vector<double> mat(2 * h->n_labels);
            for (int l = 0; l < h->n_labels; ++l) {
                mat[2 * l] = h->table[l].n;
                mat[2 * l + 1] = h->table[l].k;
            }
            ACK(cudaMalloc(&d_mat, mat.size() * sizeof(double)));
            ACK(cudaMemcpy(d_mat, mat.data(), mat.size() * sizeof(double), cudaMemcpyHostToDevice));
            ACK(cudaMalloc(&d_gl, mat.size() * sizeof(double)));
            ACK(cudaMemsetAsync(d_gl, 0, mat.size() * sizeof(double), h->stream));
            ch.mat = d_mat;
            ch.g_lab = d_gl;
        }
        k_adj_chain<<<grd, blk, 0, h->stream>>>(ch);
        h->total_launches += 1;
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess && g_eps)
            e = cudaMemcpy(g_eps, d_ge, cells * sizeof(double), cudaMemcpyDefault);
        if (e == cudaSuccess && g_sigma)
            e = cudaMemcpy(g_sigma, d_gs, cells * sizeof(double), cudaMemcpyDefault);
        if (e == cudaSuccess && g_label && d_gl)
            e = cudaMemcpy(g_label, d_gl, 2 * h->n_labels * sizeof(double), cudaMemcpyDefault);
        cudaFree(d_ge); cudaFree(d_gs);
        if (d_gl) cudaFree(d_gl);
        if (d_mat) cudaFree(d_mat);
        ACK(e);
        if (out) {
            out[0] = wR * R + wT * T;
            out[1] = R;
            out[2] = T;
        }
        cleanup();
        return FDTD_OK;
    } catch (const Fail& fl) {
        cleanup();
        return fl.code;
    }
}

}  // extern "C"
