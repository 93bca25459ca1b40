// Per-half-step field kernels, the empty-domain column kernel, the flux
// reduction and the field pack/unpack kernels.
#include <cuda_runtime.h>

#include <algorithm>

#include "fdtd_internal.h"

namespace fdtd {

// Centre field n-1/2 -> n+1/2 on every cell: Ez (S, Sec. 2.3 TMz Ez update)
// or F = eta0 Hz (P, TEz Hz update, loss-free coefficients (1, S)), with the
// CPML recursion in the top/bottom rows and the TF/SF correction at js.
// With a tape (S, the adjoint's recompute) it also stores the step's two
// gradient factors of each cell: Ez^{n-1/2} at tape and the factor of cb in
// the update (the curl with its CPML and TF/SF terms) at tape + tape_f.
template <int POL>
__global__ void k_naive_e(StepArgs a, float* __restrict__ ez, const float* __restrict__ hx,
                          const float* __restrict__ hy, float* __restrict__ psiE, int64_t n,
                          float* __restrict__ tape, size_t tape_f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= a.nx) return;
    const size_t o = (size_t)j * a.pitch + i;
    const int ir = (i + 1 == a.nx) ? 0 : i + 1;                       // periodic x
    const float dhy = __fsub_rn(hy[(size_t)j * a.pitch + ir], hy[o]);
    const float hxb = (j + 1 < a.ny) ? hx[o + a.pitch] : 0.0f;         // Hx[ny] = 0
    float dhx = __fsub_rn(hxb, hx[o]);
    if (j == a.js) dhx = __fsub_rn(dhx, tab(a.hinc, n, a));            // TF cell sees total Hx
    float2 c;
    if (POL == 0) c = a.cellcoef ? a.cellcoef[o] : coef_at(a, a.labels[(size_t)j * a.lpitch + i]);
    else c = make_float2(1.0f, a.S);
    const float e = ez[o];
    const int pj = pml_e_index(j, a.ny, a.P);
    if (pj >= 0) {
        const float b = a.pml_e[pj], cc = a.pml_e[2 * a.P + pj], ik = a.pml_e[4 * a.P + pj];
        float* pp = psiE + (size_t)pj * a.pitch + i;
        const float p = psi_new(b, cc, *pp, dhx);
        *pp = p;
        ez[o] = ez_new_pml(c.x, c.y, e, dhy, dhx, ik, p);
        if (tape) {
            tape[o] = e;
            tape[tape_f + o] = __fadd_rn(dhy, __fmaf_rn(dhx, ik, p));
        }
    } else {
        ez[o] = ez_new(c.x, c.y, e, dhy, dhx);
        if (tape) {
            tape[o] = e;
            tape[tape_f + o] = __fadd_rn(dhy, dhx);
        }
    }
}

// Edge fields n -> n+1: Hx, Hy (S, TMz updates, coefficient S) or X = -Ex,
// Y = -Ey (P, TEz updates, lossy coefficients of each edge's label pair).
// Row 0 of the top-edge field stays 0.
template <int POL>
__global__ void k_naive_h(StepArgs a, const float* __restrict__ ez, float* __restrict__ hx,
                          float* __restrict__ hy, float* __restrict__ psiH, int64_t n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= a.nx) return;
    const size_t o = (size_t)j * a.pitch + i;
    const int il = (i == 0) ? a.nx - 1 : i - 1;                        // periodic x
    const float e = ez[o];
    const size_t lo = (size_t)j * a.lpitch;
    if (POL == 0) {
        hy[o] = h_new(hy[o], a.S, __fsub_rn(e, ez[(size_t)j * a.pitch + il]));
    } else {
        const float2 cy = coef_at(a, pair_index(a.labels[lo + il], a.labels[lo + i]));
        hy[o] = e_edge_new(cy.x, cy.y, hy[o], __fsub_rn(e, ez[(size_t)j * a.pitch + il]));
    }
    if (j > 0) {
        float d = __fsub_rn(e, ez[o - a.pitch]);
        if (j == a.js) d = __fsub_rn(d, tab(a.einc, n, a));            // SF edge sees scattered Ez
        float2 cx = make_float2(1.0f, a.S);
        if (POL == 1) cx = coef_at(a, pair_index(a.labels[lo - a.lpitch + i], a.labels[lo + i]));
        const int pj = pml_h_index(j, a.ny, a.P);
        if (pj >= 0) {
            const float b = a.pml_h[pj], cc = a.pml_h[2 * a.P + pj], ik = a.pml_h[4 * a.P + pj];
            float* pp = psiH + (size_t)pj * a.pitch + i;
            const float p = psi_new(b, cc, *pp, d);
            *pp = p;
            hx[o] = (POL == 0) ? h_new_pml(hx[o], a.S, d, ik, p)
                               : e_edge_new_pml(cx.x, cx.y, hx[o], d, ik, p);
        } else {
            hx[o] = (POL == 0) ? h_new(hx[o], a.S, d) : e_edge_new(cx.x, cx.y, hx[o], d);
        }
    }
}

// Running DFT of the monitor rows after step n (Sec. 2.6); in P polarisation
// the same buffers hold eta0 Hz and -Ex.
__global__ void k_naive_dft(StepArgs a, const float* __restrict__ ez,
                            const float* __restrict__ hx, int64_t n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nx) return;
    const int w = blockIdx.y;
    const int row = w ? a.jt : a.jr;
    const size_t o = (size_t)row * a.pitch + i;
    dft_add(&a.dft[(size_t)(2 * w) * a.nx + i], ez[o], tab(a.phE, n, a));
    dft_add(&a.dft[(size_t)(2 * w + 1) * a.nx + i], hx_avg(hx[o], hx[o + a.pitch]),
            tab(a.phH, n, a));
}

void launch_naive_step(const StepArgs& a, float* ez, float* hx, float* hy, float* psiE,
                       float* psiH, int64_t n, cudaStream_t st, float* tape, size_t tape_f) {
    dim3 blk(256);
    dim3 grd((a.nx + 255) / 256, a.ny);
    if (a.pol == 0) {
        k_naive_e<0><<<grd, blk, 0, st>>>(a, ez, hx, hy, psiE, n, tape, tape_f);
        k_naive_h<0><<<grd, blk, 0, st>>>(a, ez, hx, hy, psiH, n);
    } else {
        k_naive_e<1><<<grd, blk, 0, st>>>(a, ez, hx, hy, psiE, n, nullptr, 0);
        k_naive_h<1><<<grd, blk, 0, st>>>(a, ez, hx, hy, psiH, n);
    }
    k_naive_dft<<<dim3((a.nx + 255) / 256, 2), blk, 0, st>>>(a, ez, hx, n);
}

// Empty-domain reference run: one column of air (an x-uniform field has
// Hy = 0 and needs a single column), same rows, CPML, source and monitors.
// One block advances `steps` steps; the column lives in global memory.
__device__ __forceinline__ void twin_column_global(const TwinArgs& a, int64_t n0, int steps) {
    const int ny = a.ny;
    for (int s = 0; s < steps; ++s) {
        const int64_t n = n0 + s;
        const float hinc = tab_n(a.hinc, n, a.n_tab, a.dbg), einc = tab_n(a.einc, n, a.n_tab, a.dbg);
        for (int j = threadIdx.x; j < ny; j += blockDim.x) {
            const float hxb = (j + 1 < ny) ? a.hx[j + 1] : 0.0f;
            float dhx = __fsub_rn(hxb, a.hx[j]);
            if (j == a.js) dhx = __fsub_rn(dhx, hinc);
            const float e = a.ez[j];
            const int pj = pml_e_index(j, ny, a.P);
            if (pj >= 0) {
                const float p = psi_new(a.pml_e[pj], a.pml_e[2 * a.P + pj], a.psiE[pj], dhx);
                a.psiE[pj] = p;
                a.ez[j] = ez_new_pml(a.ca, a.cb, e, 0.0f, dhx, a.pml_e[4 * a.P + pj], p);
            } else {
                a.ez[j] = ez_new(a.ca, a.cb, e, 0.0f, dhx);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            dft_add(&a.dft[0], a.ez[a.jr], tab_n(a.phE, n, a.n_tab, a.dbg));
            dft_add(&a.dft[2], a.ez[a.jt], tab_n(a.phE, n, a.n_tab, a.dbg));
        }
        for (int j = threadIdx.x + 1; j < ny; j += blockDim.x) {
            float d = __fsub_rn(a.ez[j], a.ez[j - 1]);
            if (j == a.js) d = __fsub_rn(d, einc);
            const int pj = pml_h_index(j, ny, a.P);
            if (pj >= 0) {
                const float p = psi_new(a.pml_h[pj], a.pml_h[2 * a.P + pj], a.psiH[pj], d);
                a.psiH[pj] = p;
                a.hx[j] = h_new_pml(a.hx[j], a.S, d, a.pml_h[4 * a.P + pj], p);
            } else {
                a.hx[j] = h_new(a.hx[j], a.S, d);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            dft_add(&a.dft[1], hx_avg(a.hx[a.jr], a.hx[a.jr + 1]), tab_n(a.phH, n, a.n_tab, a.dbg));
            dft_add(&a.dft[3], hx_avg(a.hx[a.jt], a.hx[a.jt + 1]), tab_n(a.phH, n, a.n_tab, a.dbg));
        }
    }
}

__global__ void __launch_bounds__(1024) k_twin(TwinArgs a, int64_t n0, int steps) {
    twin_column_global(a, n0, steps);
}

// The same column kept in shared memory for the whole launch (when it fits):
// identical arithmetic and order, the DFT sums carried in registers of
// thread 0 and written back at the end.
__device__ __forceinline__ void twin_column_smem(const TwinArgs& a, int64_t n0, int steps,
                                                 float* sm) {
    const int ny = a.ny, P2 = 2 * a.P;
    float* ez = sm;
    float* hx = sm + ny;
    float* pE = hx + ny;
    float* pH = pE + P2;
    for (int j = threadIdx.x; j < ny; j += blockDim.x) { ez[j] = a.ez[j]; hx[j] = a.hx[j]; }
    for (int j = threadIdx.x; j < P2; j += blockDim.x) { pE[j] = a.psiE[j]; pH[j] = a.psiH[j]; }
    double2 d0 = a.dft[0], d1 = a.dft[1], d2 = a.dft[2], d3 = a.dft[3];
    __syncthreads();
    for (int s = 0; s < steps; ++s) {
        const int64_t n = n0 + s;
        const float hinc = tab_n(a.hinc, n, a.n_tab, a.dbg), einc = tab_n(a.einc, n, a.n_tab, a.dbg);
        for (int j = threadIdx.x; j < ny; j += blockDim.x) {
            const float hxb = (j + 1 < ny) ? hx[j + 1] : 0.0f;
            float dhx = __fsub_rn(hxb, hx[j]);
            if (j == a.js) dhx = __fsub_rn(dhx, hinc);
            const float e = ez[j];
            const int pj = pml_e_index(j, ny, a.P);
            if (pj >= 0) {
                const float p = psi_new(a.pml_e[pj], a.pml_e[2 * a.P + pj], pE[pj], dhx);
                pE[pj] = p;
                ez[j] = ez_new_pml(a.ca, a.cb, e, 0.0f, dhx, a.pml_e[4 * a.P + pj], p);
            } else {
                ez[j] = ez_new(a.ca, a.cb, e, 0.0f, dhx);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            dft_add(&d0, ez[a.jr], tab_n(a.phE, n, a.n_tab, a.dbg));
            dft_add(&d2, ez[a.jt], tab_n(a.phE, n, a.n_tab, a.dbg));
        }
        for (int j = threadIdx.x + 1; j < ny; j += blockDim.x) {
            float d = __fsub_rn(ez[j], ez[j - 1]);
            if (j == a.js) d = __fsub_rn(d, einc);
            const int pj = pml_h_index(j, ny, a.P);
            if (pj >= 0) {
                const float p = psi_new(a.pml_h[pj], a.pml_h[2 * a.P + pj], pH[pj], d);
                pH[pj] = p;
                hx[j] = h_new_pml(hx[j], a.S, d, a.pml_h[4 * a.P + pj], p);
            } else {
                hx[j] = h_new(hx[j], a.S, d);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            dft_add(&d1, hx_avg(hx[a.jr], hx[a.jr + 1]), tab_n(a.phH, n, a.n_tab, a.dbg));
            dft_add(&d3, hx_avg(hx[a.jt], hx[a.jt + 1]), tab_n(a.phH, n, a.n_tab, a.dbg));
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < ny; j += blockDim.x) { a.ez[j] = ez[j]; a.hx[j] = hx[j]; }
    for (int j = threadIdx.x; j < P2; j += blockDim.x) { a.psiE[j] = pE[j]; a.psiH[j] = pH[j]; }
    if (threadIdx.x == 0) { a.dft[0] = d0; a.dft[1] = d1; a.dft[2] = d2; a.dft[3] = d3; }
}

__global__ void __launch_bounds__(512) k_twin_smem(TwinArgs a, int64_t n0, int steps) {
    extern __shared__ float sm[];
    twin_column_smem(a, n0, steps, sm);
}

// One block per simulation of a batch; steps start at n_base + *step_base.
__global__ void __launch_bounds__(512) k_twin_batch_smem(const TwinArgs* tws,
                                                         const int64_t* step_base, int steps) {
    extern __shared__ float sm[];
    const TwinArgs a = tws[blockIdx.x];
    twin_column_smem(a, a.n_base + *step_base, steps, sm);
}

__global__ void __launch_bounds__(1024) k_twin_batch_global(const TwinArgs* tws,
                                                            const int64_t* step_base, int steps) {
    const TwinArgs a = tws[blockIdx.x];
    twin_column_global(a, a.n_base + *step_base, steps);
}

void launch_twin(const TwinArgs& a, int64_t n0, int steps, cudaStream_t st) {
    constexpr size_t kMaxSmem = 200 * 1024;
    const size_t smem = (size_t)(2 * a.ny + 4 * a.P) * sizeof(float);
    if (smem <= kMaxSmem) {
        static bool configured[64] = {};   // the opt-in is per function and device
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64 || !configured[dev]) {
            cudaFuncSetAttribute(k_twin_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxSmem);
            if (dev >= 0 && dev < 64) configured[dev] = true;
        }
        k_twin_smem<<<1, 512, smem, st>>>(a, n0, steps);
    } else {
        k_twin<<<1, 1024, 0, st>>>(a, n0, steps);
    }
}

// Shared-memory opt-in of the batched column kernel on the current device;
// done before any stream capture that contains the kernel.
void configure_twin_batch() {
    cudaFuncSetAttribute(k_twin_batch_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
}

void launch_twin_batch(const TwinArgs* tws, int n, int max_ny, int max_P,
                       const int64_t* step_base, int steps, cudaStream_t st) {
    constexpr size_t kMaxSmem = 200 * 1024;
    const size_t smem = (size_t)(2 * max_ny + 4 * max_P) * sizeof(float);
    if (smem <= kMaxSmem) {
        static bool configured[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64 || !configured[dev]) {
            cudaFuncSetAttribute(k_twin_batch_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxSmem);
            if (dev >= 0 && dev < 64) configured[dev] = true;
        }
        k_twin_batch_smem<<<n, 512, smem, st>>>(tws, step_base, steps);
    } else {
        k_twin_batch_global<<<n, 1024, 0, st>>>(tws, step_base, steps);
    }
}

// Flux sums (Sec. 2.6, Poynting form): out[0] = sum_i Re(E_r conj(H_r)),
// out[1] = sum_i Re(E_t conj(H_t)), out[2] = Re(E_t conj(H_t)) of the empty
// column. Warp-shuffle then shared-memory reduction in a fixed order.
__global__ void __launch_bounds__(1024) k_flux(const double2* __restrict__ dft,
                                               const double2* __restrict__ tw, int nx,
                                               double* out) {
    __shared__ double sh[2][32];
    double ar = 0.0, at = 0.0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const double2 er = dft[i], hr = dft[nx + i], et = dft[2 * nx + i], ht = dft[3 * nx + i];
        ar += er.x * hr.x + er.y * hr.y;
        at += et.x * ht.x + et.y * ht.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_down_sync(0xffffffffu, ar, o);
        at += __shfl_down_sync(0xffffffffu, at, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[0][w] = ar; sh[1][w] = at; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        ar = (l < nw) ? sh[0][l] : 0.0;
        at = (l < nw) ? sh[1][l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            ar += __shfl_down_sync(0xffffffffu, ar, o);
            at += __shfl_down_sync(0xffffffffu, at, o);
        }
        if (l == 0) {
            out[0] = ar;
            out[1] = at;
            out[2] = tw[2].x * tw[3].x + tw[2].y * tw[3].y;
        }
    }
}

void launch_flux(const double2* dft, const double2* twin_dft, int nx, double* out,
                 cudaStream_t st) {
    k_flux<<<1, 1024, 0, st>>>(dft, twin_dft, nx, out);
}

// Bloch-order amplitudes of the four monitor lines (Sec. 2.6): block o
// computes, for m = o - m_max, X_m = (1/nx) sum_i X_i exp(-2 pi i m i / nx)
// for each line X in FP64. The phase index m i is reduced modulo nx in
// integers before sincospi, so the twiddles are exact to rounding.
__global__ void __launch_bounds__(256) k_bloch(const double2* __restrict__ dft, int nx,
                                               int m_max, double2* __restrict__ out) {
    __shared__ double2 sh[4][8];
    const int o = blockIdx.x;
    const int64_t m = (int64_t)o - m_max;
    const int64_t mm = ((m % nx) + nx) % nx;
    double2 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int64_t r = (mm * i) % nx;
        double sn, cs;
        sincospi(2.0 * (double)r / (double)nx, &sn, &cs);      // e^{-i theta} = cs - i sn
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 v = dft[(size_t)q * nx + i];
            acc[q].x = fma(v.x, cs, fma(v.y, sn, acc[q].x));
            acc[q].y = fma(v.y, cs, fma(-v.x, sn, acc[q].y));
        }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        for (int s = 16; s > 0; s >>= 1) {
            acc[q].x += __shfl_down_sync(0xffffffffu, acc[q].x, s);
            acc[q].y += __shfl_down_sync(0xffffffffu, acc[q].y, s);
        }
        if (l == 0) sh[q][w] = acc[q];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int q = threadIdx.x;
        double2 t = make_double2(0.0, 0.0);
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { t.x += sh[q][k].x; t.y += sh[q][k].y; }
        out[(size_t)q * (2 * m_max + 1) + o] = make_double2(t.x / nx, t.y / nx);
    }
}

void launch_bloch(const double2* dft, int nx, int m_max, double2* out, cudaStream_t st) {
    k_bloch<<<2 * m_max + 1, 256, 0, st>>>(dft, nx, m_max, out);
}

__global__ void k_pack(const float* __restrict__ src, int pitch, int nx, int ny, float scale,
                       float* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < nx) dst[(size_t)j * nx + i] = src[(size_t)j * pitch + i] * scale;
}

__global__ void k_unpack(const float* __restrict__ src, int nx, int ny, float scale,
                         float* __restrict__ dst, int pitch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < nx) dst[(size_t)j * pitch + i] = src[(size_t)j * nx + i] * scale;
}

void launch_pack(const float* src, int pitch, int nx, int ny, float scale, float* dst,
                 cudaStream_t st) {
    k_pack<<<dim3((nx + 255) / 256, ny), 256, 0, st>>>(src, pitch, nx, ny, scale, dst);
}

void launch_unpack(const float* src, int nx, int ny, float scale, float* dst, int pitch,
                   cudaStream_t st) {
    k_unpack<<<dim3((nx + 255) / 256, ny), 256, 0, st>>>(src, nx, ny, scale, dst, pitch);
}

__global__ void k_scale_double(double* p, int64_t n, double s) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] *= s;
}

void launch_scale_double(double* p, int64_t n, double scale, cudaStream_t st) {
    if (n > 0) k_scale_double<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, n, scale);
}

// Watchdog: sets *flag when any Ez value is not finite.
__global__ void k_check_finite(const float* __restrict__ p, int pitch, int nx, int ny,
                               int* flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < nx && !isfinite(p[(size_t)j * pitch + i])) atomicOr(flag, 1);
}

void launch_check_finite(const float* p, int pitch, int nx, int ny, int* flag,
                         cudaStream_t st) {
    k_check_finite<<<dim3((nx + 255) / 256, ny), 256, 0, st>>>(p, pitch, nx, ny, flag);
}

// Debug builds: bytes [p, p + n) must all equal `want` (a guard band);
// otherwise bit `bit` of *flag is set.
__global__ void k_guard_check(const unsigned char* p, size_t n, unsigned char want,
                              unsigned* flag, unsigned bit) {
    bool bad = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        bad |= (p[i] != want);
    if (bad) atomicOr(flag, 1u << bit);
}

void launch_guard_check(const unsigned char* p, size_t n, unsigned char want, unsigned* flag,
                        unsigned bit, cudaStream_t st) {
    if (n == 0) return;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 64);
    k_guard_check<<<blocks, 256, 0, st>>>(p, n, want, flag, bit);
}

}  // namespace fdtd
