// Temporally blocked TMz stencil: K leapfrog steps per launch.
//
// Work unit: one warp owns a strip of 128 columns (4 per lane, loaded and
// stored as float4) and a segment of rows [y0, y1). It streams down the rows
// once; at iteration t it loads level-0 row t and, for k = 0..K-1, advances
// level k to level k+1 at row t-k-1 (each level lags the one below it by one
// row, which is exactly the reach of one Yee step in s). The rows of the
// intermediate levels never leave registers: per level a lane keeps the one
// pending row (Ez, Hx, Hy and its 4 labels). Only level 0 is read from and
// level K written to memory (ping-pong buffers), so the DRAM traffic per
// cell-update falls from 25 bytes to about 25/K plus the halo overhead.
//
// Halos: one step moves information one column and one row each way, so a
// strip computes K (rounded up to 4) extra columns on each side and a
// segment K extra rows above and below; only the interior is stored.
// Columns wrap modulo nx (periodic x, Sec. 2.4); the neighbour column of
// the lane's outer column comes from the adjacent lane by shuffle.
//
// CPML rows (top/bottom P rows) carry their psi recursion from level to
// level in a per-strip scratch area; the segment plan guarantees that only
// the first and last segment of a strip ever touch CPML rows. The TF/SF
// corrections (Sec. 2.5) are applied by every segment that computes row js;
// DFT accumulation (Sec. 2.6) is done by the segment owning the monitor row,
// which the plan keeps at least one row above its segment's end.
#include <cuda_runtime.h>

#include "fdtd_internal.h"

namespace fdtd {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void ld4_rw(const float* p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

}  // namespace

template <int K>
__global__ void __launch_bounds__(128) k_blocked(const BlockedArgs a, const int64_t n0) {
    constexpr int H = ((K + 3) / 4) * 4;
    __shared__ float2 s_coef[256];
    for (int t = threadIdx.x; t < a.s.n_labels; t += blockDim.x) s_coef[t] = a.s.coef[t];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (task >= a.n_tasks) return;                 // whole warps leave together
    const int strip = task % a.n_strips;
    const int seg = task / a.n_strips;
    const int y0 = a.seg_y0[seg], y1 = a.seg_y0[seg + 1];
    const int nx = a.s.nx, ny = a.s.ny, P = a.s.P;
    const size_t pitch = (size_t)a.s.pitch;
    const size_t lpitch = (size_t)a.s.lpitch;
    const float S = a.s.S;
    const int xl = 4 * lane;                        // local column of the lane
    const int xg_pre = strip * a.w_int - H + xl;    // global column before wrapping
    const int gx = ((xg_pre % nx) + nx) % nx;       // nx % 4 == 0: 4 columns stay contiguous
    const bool own = (xl >= H) && (xl < H + a.w_int) && (xg_pre < nx);
    const bool own_r = (a.s.jr >= y0) && (a.s.jr < y1);
    const bool own_t = (a.s.jt >= y0) && (a.s.jt < y1);
    float* slotE = a.slotE + (size_t)strip * 2 * P * 128 + xl;
    float* slotH = a.slotH + (size_t)strip * 2 * P * 128 + xl;

    float pE[K + 1][4], pX[K + 1][4], pY[K][4];
    uint32_t pL[K];
#pragma unroll
    for (int k = 0; k <= K; ++k) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            pE[k][q] = 0.f; pX[k][q] = 0.f;
            if (k < K) pY[k][q] = 0.f;
        }
        if (k < K) pL[k] = 0u;
    }

    const int t_begin = (y0 == 0) ? 0 : (y0 - K);
    const int t_end = y1 + K;
    for (int t = t_begin; t < t_end; ++t) {
        float fE[4], fX[4], fY[4];
        uint32_t fL;
        if (t < ny) {
            const size_t o = (size_t)t * pitch + gx;
            ld4(a.ez_in + o, fE);
            ld4(a.hx_in + o, fX);
            ld4(a.hy_in + o, fY);
            fL = __ldg(reinterpret_cast<const uint32_t*>(a.s.labels + (size_t)t * lpitch + gx));
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) { fE[q] = 0.f; fX[q] = 0.f; fY[q] = 0.f; }
            fL = 0u;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int r = t - k - 1;                 // row of level k+1 made here
            const int lo = (y0 == 0) ? 0 : (y0 - K + k);
            const int hi = min(ny, y1 + K - k - 1);
            const int64_t n = n0 + k;                // absolute step of this level
            float oE[4], oX[4], oY[4];
            const uint32_t cL = pL[k];
            if (r >= lo && r < hi) {
                // ---- Ez^{n+1/2} at row r
                const float yR = __shfl_down_sync(FULL, pY[k][0], 1);
                const bool tf = (r == a.s.js);
                const float hinc = tf ? a.s.hinc[n] : 0.f;
                const int pe = pml_e_index(r, ny, P);
                if (pe >= 0) {
                    const float b = a.s.pml_e[pe], c = a.s.pml_e[2 * P + pe];
                    const float ik = a.s.pml_e[4 * P + pe];
                    float psi[4];
                    if (k == 0) ld4(a.psiE_in + (size_t)pe * pitch + gx, psi);
                    else ld4_rw(slotE + (size_t)pe * 128, psi);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 cc = s_coef[(cL >> (8 * q)) & 0xffu];
                        const float dhy = __fsub_rn(q < 3 ? pY[k][q + 1] : yR, pY[k][q]);
                        float dhx = __fsub_rn(fX[q], pX[k][q]);
                        if (tf) dhx = __fsub_rn(dhx, hinc);
                        psi[q] = psi_new(b, c, psi[q], dhx);
                        oE[q] = ez_new_pml(cc.x, cc.y, pE[k][q], dhy, dhx, ik, psi[q]);
                    }
                    if (k == K - 1) {
                        if (own) st4(a.psiE_out + (size_t)pe * pitch + gx, psi);
                    } else {
                        st4(slotE + (size_t)pe * 128, psi);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 cc = s_coef[(cL >> (8 * q)) & 0xffu];
                        const float dhy = __fsub_rn(q < 3 ? pY[k][q + 1] : yR, pY[k][q]);
                        float dhx = __fsub_rn(fX[q], pX[k][q]);
                        if (tf) dhx = __fsub_rn(dhx, hinc);
                        oE[q] = ez_new(cc.x, cc.y, pE[k][q], dhy, dhx);
                    }
                }
                // ---- Hx^{n+1} at edge r (edge 0 is fixed)
                if (r > 0) {
                    const float einc = tf ? a.s.einc[n] : 0.f;
                    const int ph = pml_h_index(r, ny, P);
                    if (ph >= 0) {
                        const float b = a.s.pml_h[ph], c = a.s.pml_h[2 * P + ph];
                        const float ik = a.s.pml_h[4 * P + ph];
                        float psi[4];
                        if (k == 0) ld4(a.psiH_in + (size_t)ph * pitch + gx, psi);
                        else ld4_rw(slotH + (size_t)ph * 128, psi);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float d = __fsub_rn(oE[q], pE[k + 1][q]);
                            if (tf) d = __fsub_rn(d, einc);
                            psi[q] = psi_new(b, c, psi[q], d);
                            oX[q] = h_new_pml(pX[k][q], S, d, ik, psi[q]);
                        }
                        if (k == K - 1) {
                            if (own) st4(a.psiH_out + (size_t)ph * pitch + gx, psi);
                        } else {
                            st4(slotH + (size_t)ph * 128, psi);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float d = __fsub_rn(oE[q], pE[k + 1][q]);
                            if (tf) d = __fsub_rn(d, einc);
                            oX[q] = h_new(pX[k][q], S, d);
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) oX[q] = pX[k][q];
                }
                // ---- Hy^{n+1} at row r
                const float eL = __shfl_up_sync(FULL, oE[3], 1);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    oY[q] = h_new(pY[k][q], S, __fsub_rn(oE[q], q > 0 ? oE[q - 1] : eL));
                // ---- monitor DFTs (Sec. 2.6) by the owning segment
                if (own) {
                    if (own_r && r == a.s.jr) {
                        const double2 ph = a.s.phE[n];
#pragma unroll
                        for (int q = 0; q < 4; ++q) dft_add(&a.s.dft[gx + q], oE[q], ph);
                    }
                    if (own_r && r == a.s.jr + 1) {
                        const double2 ph = a.s.phH[n];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            dft_add(&a.s.dft[nx + gx + q], hx_avg(pX[k + 1][q], oX[q]), ph);
                    }
                    if (own_t && r == a.s.jt) {
                        const double2 ph = a.s.phE[n];
#pragma unroll
                        for (int q = 0; q < 4; ++q) dft_add(&a.s.dft[2 * nx + gx + q], oE[q], ph);
                    }
                    if (own_t && r == a.s.jt + 1) {
                        const double2 ph = a.s.phH[n];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            dft_add(&a.s.dft[3 * nx + gx + q], hx_avg(pX[k + 1][q], oX[q]), ph);
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) { oE[q] = 0.f; oX[q] = 0.f; oY[q] = 0.f; }
            }
            // level k now waits at row r+1; the new level-(k+1) row r flows up
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                pE[k][q] = fE[q]; pX[k][q] = fX[q]; pY[k][q] = fY[q];
                fE[q] = oE[q]; fX[q] = oX[q]; fY[q] = oY[q];
            }
            pL[k] = fL;
            fL = cL;
        }
        const int ro = t - K;
        if (own && ro >= y0 && ro < y1) {
            const size_t o = (size_t)ro * pitch + gx;
            st4(a.ez_out + o, fE);
            st4(a.hx_out + o, fX);
            st4(a.hy_out + o, fY);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) { pE[K][q] = fE[q]; pX[K][q] = fX[q]; }
    }
}

int blocked_max_K() { return 8; }

bool launch_blocked(const BlockedArgs& a, int K, int64_t n0, cudaStream_t st) {
    const int warps = 4;
    const unsigned grid = (unsigned)((a.n_tasks + warps - 1) / warps);
    switch (K) {
        case 1: k_blocked<1><<<grid, 32 * warps, 0, st>>>(a, n0); break;
        case 2: k_blocked<2><<<grid, 32 * warps, 0, st>>>(a, n0); break;
        case 3: k_blocked<3><<<grid, 32 * warps, 0, st>>>(a, n0); break;
        case 4: k_blocked<4><<<grid, 32 * warps, 0, st>>>(a, n0); break;
        case 5: k_blocked<5><<<grid, 32 * warps, 0, st>>>(a, n0); break;
        case 6: k_blocked<6><<<grid, 32 * warps, 0, st>>>(a, n0); break;
        case 7: k_blocked<7><<<grid, 32 * warps, 0, st>>>(a, n0); break;
        case 8: k_blocked<8><<<grid, 32 * warps, 0, st>>>(a, n0); break;
        default: return false;
    }
    return true;
}

}  // namespace fdtd
