// Temporally blocked stencil kernels (templates): K leapfrog steps per
// launch. Instantiated by blocked_s.cu (S polarisation, single runs),
// blocked_sb.cu (S, batches) and blocked_p.cu (P); launched through the
// dispatchers of blocked.cu.
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
// P polarisation (POL = 1, TEz in the variables eta0 Hz, -Ex, -Ey) runs the
// same pipeline with loss-free centre updates and lossy edge updates whose
// coefficients come from the label pair of each edge: the top edge of row r
// pairs rows r-1 and r (level k+1 still holds the label word of row r-1 as
// its pending row; level K keeps one extra word), the left edge of column q
// pairs columns q-1 and q (the neighbour lane's last label by shuffle).
//
// CPML rows (top/bottom P rows) carry their psi recursion from level to
// level in a per-warp shared-memory ring; any segment may hold CPML rows,
// and only the segment owning a row stores its psi (like its fields). The
// TF/SF corrections (Sec. 2.5) are applied by every segment that computes
// row js; DFT accumulation (Sec. 2.6) is done by the segment owning the
// monitor row, which the plan keeps at least one row above its segment's
// end. Every segment but the first starts at row K or later, so its halo
// rows exist.
#pragma once
#include <cuda_runtime.h>

#include "fdtd_internal.h"

namespace fdtd {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// The four columns of a lane as two register pairs, columns (0, 1) and
// (2, 3), so that paired FP32 instructions take them without moves; v[q]
// names column q.
struct V4 {
    float2 a, b;
    __device__ __forceinline__ float& operator[](int q) {
        return q < 2 ? (q == 0 ? a.x : a.y) : (q == 2 ? b.x : b.y);
    }
    __device__ __forceinline__ float operator[](int q) const {
        return q < 2 ? (q == 0 ? a.x : a.y) : (q == 2 ? b.x : b.y);
    }
};
__device__ __forceinline__ void ld4(const float* p, V4& v) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v.a = make_float2(x.x, x.y); v.b = make_float2(x.z, x.w);
}
__device__ __forceinline__ void st4(float* p, const V4& v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.a.x, v.a.y, v.b.x, v.b.y);
}
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Asynchronous global -> shared copies (cp.async); `bytes` = 0 zero-fills the
// destination without reading the source.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kRing = 4;   // rows in flight per warp for code shape 2

}  // namespace

// Register state of one warp's pipeline: per level k the pending row
// (Ez, Hx, Hy, 4 packed labels); level K keeps Ez and Hx of its last row
// (and, for POL = 1, its label word).
template <int K>
struct Pipe {
    V4 E[K + 1], X[K + 1], Y[K];
    uint32_t L[K + 1];
    uint32_t LY[K];   // P, code shape 5: left-edge label pairs of the pending row
};

struct Lane {
    const float2* coef;
    const float4* pair;   // code shape 5: label-pair table (shared memory)
    int gx, y0, y1, ny, P, nx;
    bool own, own_r, own_t;
    bool col_ok;          // the lane's 4 columns lie in [0, nx) (debug index check)
    float S;
};

// Code shape 5 (S polarisation, at most 16 labels) keeps, in place of the
// packed label word of a row, the byte offsets of the label-pair table
// entries of the lane's column pairs (0, 1) and (2, 3), 16 bits each. Entry
// b0 | b1 << 4 holds (ca[b0], ca[b1], cb[b0], cb[b1]), the coefficients of
// two neighbouring cells with labels b0 and b1 as two register pairs.
__device__ __forceinline__ uint32_t pair_offsets(uint32_t w) {
    return ((w | (w >> 4)) & 0x00ff00ffu) << 4;
}
__device__ __forceinline__ float4 pair_at(const float4* tab, uint32_t off) {
    return *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(tab) + off);
}

// Code shapes with the paired FP32 lean path (5 and 6, at most 16 labels);
// for S polarisation their coefficients come from the label-pair table.
template <int V>
constexpr bool kPairShape = (V == 5 || V == 6);

// S: (ca, cb) of column q of a lane from its row's label word.
template <int V>
__device__ __forceinline__ float2 coef_s(const Lane& ln, uint32_t w, int q) {
    if (kPairShape<V>) {
        const float4 c = pair_at(ln.pair, q < 2 ? (w & 0xffffu) : (w >> 16));
        return (q & 1) ? make_float2(c.y, c.w) : make_float2(c.x, c.z);
    }
    return ln.coef[(w >> (8 * q)) & 0xffu];
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Lean S iteration of code shape 5 with paired FP32 instructions
// (fma/add/mul .f32x2): a lane's columns (0, 1) and (2, 3) form the pairs.
// Each element of a paired instruction rounds exactly as the scalar _rn
// intrinsic, and a - b is formed as fma(b, -1, a), which rounds like a
// subtraction, so the results are bit for bit those of advance(). The
// differences along x take a column pair shifted by one and stay scalar.
template <int K, int V>
__device__ __forceinline__ void lean_pair_level(Pipe<K>& p, const int k, V4& fE, V4& fX,
                                                V4& fY, uint32_t& fL, const Lane& ln,
                                                const BlockedArgs& a, const int t) {
    const float2 S2 = f2(ln.S, ln.S);
    const float2 M1 = f2(-1.0f, -1.0f);
    {
        const uint32_t cL = p.L[k];
        const float4 c01 = pair_at(ln.pair, cL & 0xffffu);
        const float4 c23 = pair_at(ln.pair, cL >> 16);
        const float yR = __shfl_down_sync(FULL, p.Y[k][0], 1);
        const float2 dhx01 = __ffma2_rn(p.X[k].a, M1, fX.a);
        const float2 dhx23 = __ffma2_rn(p.X[k].b, M1, fX.b);
        const float2 dhy01 = f2(__fsub_rn(p.Y[k][1], p.Y[k][0]), __fsub_rn(p.Y[k][2], p.Y[k][1]));
        const float2 dhy23 = f2(__fsub_rn(p.Y[k][3], p.Y[k][2]), __fsub_rn(yR, p.Y[k][3]));
        const float2 cu01 = __fadd2_rn(dhy01, dhx01);
        const float2 cu23 = __fadd2_rn(dhy23, dhx23);
        const float2 e01 = __ffma2_rn(f2(c01.z, c01.w), cu01, __fmul2_rn(f2(c01.x, c01.y), p.E[k].a));
        const float2 e23 = __ffma2_rn(f2(c23.z, c23.w), cu23, __fmul2_rn(f2(c23.x, c23.y), p.E[k].b));
        if (V == 6) {
            // code shape 6: step n0+k's gradient factors of this row (adjoint tape)
            const int r = t - k - 1;
            if (ln.own && r >= ln.y0 && r < ln.y1) {
                float* tp = a.tape[k] + (size_t)r * a.s.pitch + ln.gx;
                st4(tp, p.E[k]);
                *reinterpret_cast<float4*>(tp + a.tape_f) = make_float4(cu01.x, cu01.y, cu23.x, cu23.y);
            }
        }
        const float2 d01 = __ffma2_rn(p.E[k + 1].a, M1, e01);
        const float2 d23 = __ffma2_rn(p.E[k + 1].b, M1, e23);
        const float2 x01 = __ffma2_rn(S2, d01, p.X[k].a);
        const float2 x23 = __ffma2_rn(S2, d23, p.X[k].b);
        const float eL = __shfl_up_sync(FULL, e23.y, 1);
        const float2 dy01 = f2(__fsub_rn(e01.x, eL), __fsub_rn(e01.y, e01.x));
        const float2 dy23 = f2(__fsub_rn(e23.x, e01.y), __fsub_rn(e23.y, e23.x));
        const float2 y01 = __ffma2_rn(S2, dy01, p.Y[k].a);
        const float2 y23 = __ffma2_rn(S2, dy23, p.Y[k].b);
        // level k now waits at row r+1; the new level-(k+1) row r flows up
        p.E[k] = fE; p.X[k] = fX; p.Y[k] = fY;
        fE.a = e01; fE.b = e23;
        fX.a = x01; fX.b = x23;
        fY.a = y01; fY.b = y23;
        p.L[k] = fL;
        fL = cL;
    }
}

template <int K, int V>
__device__ __forceinline__ void advance_lean_pair(Pipe<K>& p, V4& fE, V4& fX,
                                                  V4& fY, uint32_t& fL, const Lane& ln,
                                                  const BlockedArgs& a, const int t) {
#pragma unroll
    for (int k = 0; k < K; ++k) lean_pair_level<K, V>(p, k, fE, fX, fY, fL, ln, a, t);
}

// Lean P iteration of code shape 5: the same pipeline as advance() for
// POL = 1 with the loss-free centre update and the two edge differences
// along s paired (f32x2); the centre's coefficient 1 is dropped (1 * F is F
// exactly) and the lossy edge updates keep their per-edge label-pair
// coefficients (scalar). Bit for bit the results of advance().
template <int K>
__device__ __forceinline__ void lean_pair_p_level(Pipe<K>& p, const int k, V4& fE, V4& fX,
                                                  V4& fY, uint32_t& fL, uint32_t& fLY,
                                                  const Lane& ln) {
    const float2 S2 = f2(ln.S, ln.S);
    const float2 M1 = f2(-1.0f, -1.0f);
    {
        // the row's edge label pairs, formed once when the row was loaded
        const uint32_t xP = p.L[k], yP = p.LY[k];
        const float yR = __shfl_down_sync(FULL, p.Y[k][0], 1);
        const float2 dhx01 = __ffma2_rn(p.X[k].a, M1, fX.a);
        const float2 dhx23 = __ffma2_rn(p.X[k].b, M1, fX.b);
        const float2 dhy01 = f2(__fsub_rn(p.Y[k][1], p.Y[k][0]), __fsub_rn(p.Y[k][2], p.Y[k][1]));
        const float2 dhy23 = f2(__fsub_rn(p.Y[k][3], p.Y[k][2]), __fsub_rn(yR, p.Y[k][3]));
        const float2 e01 = __ffma2_rn(S2, __fadd2_rn(dhy01, dhx01), p.E[k].a);
        const float2 e23 = __ffma2_rn(S2, __fadd2_rn(dhy23, dhx23), p.E[k].b);
        const float2 d01 = __ffma2_rn(p.E[k + 1].a, M1, e01);
        const float2 d23 = __ffma2_rn(p.E[k + 1].b, M1, e23);
        const float oE[4] = {e01.x, e01.y, e23.x, e23.y};
        const float d[4] = {d01.x, d01.y, d23.x, d23.y};
        float oX[4], oY[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 cx = ln.coef[(xP >> (8 * q)) & 0xffu];
            oX[q] = e_edge_new(cx.x, cx.y, p.X[k][q], d[q]);
        }
        const float eL = __shfl_up_sync(FULL, oE[3], 1);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float dy = __fsub_rn(oE[q], q > 0 ? oE[q - 1] : eL);
            const float2 cy = ln.coef[(yP >> (8 * q)) & 0xffu];
            oY[q] = e_edge_new(cy.x, cy.y, p.Y[k][q], dy);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            p.E[k][q] = fE[q]; p.X[k][q] = fX[q]; p.Y[k][q] = fY[q];
            fE[q] = oE[q]; fX[q] = oX[q]; fY[q] = oY[q];
        }
        p.L[k] = fL;
        fL = xP;
        p.LY[k] = fLY;
        fLY = yP;
    }
}

template <int K>
__device__ __forceinline__ void advance_lean_pair_p(Pipe<K>& p, V4& fE, V4& fX,
                                                    V4& fY, uint32_t& fL, uint32_t& fLY,
                                                    const Lane& ln) {
#pragma unroll
    for (int k = 0; k < K; ++k) lean_pair_p_level<K>(p, k, fE, fX, fY, fL, fLY, ln);
}

// Two lean rows t and t+1 of code shape 5 in one pass over the levels,
// row t+1 one level behind row t: level k of row t+1 needs level k of row t
// (its pending rows) and level k-1 of row t+1, so at stage s the code
// holds level s of row t and level s-1 of row t+1, two independent chains.
// Row t leaves the pipeline (finish0: its level-K row stored, level K's
// pending row set) before row t+1's last level reads it. The same
// per-level expressions in an order that keeps every dependency, so the
// same bits.
template <int K, int V, int POL>
__device__ __forceinline__ void lean_level5(Pipe<K>& p, const int k, V4& fE, V4& fX, V4& fY,
                                            uint32_t& fL, uint32_t& fLY, const Lane& ln,
                                            const BlockedArgs& a, const int t) {
    if constexpr (POL == 0) lean_pair_level<K, V>(p, k, fE, fX, fY, fL, ln, a, t);
    else lean_pair_p_level<K>(p, k, fE, fX, fY, fL, fLY, ln);
}

template <int K, int V, int POL, typename F>
__device__ __forceinline__ void advance_lean_pair2(Pipe<K>& p, V4& fE0, V4& fX0, V4& fY0,
                                                   uint32_t& fL0, uint32_t& fLY0, V4& fE1,
                                                   V4& fX1, V4& fY1, uint32_t& fL1,
                                                   uint32_t& fLY1, const Lane& ln,
                                                   const BlockedArgs& a, const int t,
                                                   F&& finish0) {
#pragma unroll
    for (int s = 0; s <= K; ++s) {
        if (s < K) lean_level5<K, V, POL>(p, s, fE0, fX0, fY0, fL0, fLY0, ln, a, t);
        if (s == K) finish0();
        if (s >= 1) lean_level5<K, V, POL>(p, s - 1, fE1, fX1, fY1, fL1, fLY1, ln, a, t + 1);
    }
}

// One iteration of the pipeline: level k advances at row t-k-1, k = 0..K-1.
// GENERAL = false is the lean path for iterations whose K rows hold no
// CPML, source, monitor or boundary row and lie inside the valid range;
// both paths round identically.
template <int K, bool GENERAL, int POL, int V>
__device__ __forceinline__ void advance(Pipe<K>& p, V4& fE, V4& fX,
                                        V4& fY, uint32_t& fL, uint32_t& fLY, const int t,
                                        const BlockedArgs& a, const Lane& ln, float4* ringE,
                                        float4* ringH, const int64_t n0) {
    if constexpr (!GENERAL && kPairShape<V> && POL == 0) {
        advance_lean_pair<K, V>(p, fE, fX, fY, fL, ln, a, t);
        return;
    }
    if constexpr (!GENERAL && kPairShape<V> && POL == 1) {
        advance_lean_pair_p<K>(p, fE, fX, fY, fL, fLY, ln);
        return;
    }
    const float S = ln.S;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int r = t - k - 1;
        float oE[4], oX[4], oY[4];
        float cu[4];   // code shapes 4, 6: the factor of cb in the Ez update (adjoint tape)
        const uint32_t cL = p.L[k];
        // P: packed label-pair indices (labels < 16) of the top and left edges
        uint32_t xP = 0u, yP = 0u;
        if (POL == 1 && kPairShape<V>) {
            xP = cL;                        // formed when the row was loaded
            yP = p.LY[k];
        } else if (POL == 1) {
            const uint32_t lUp = p.L[k + 1];                          // row r-1
            const uint32_t lNb = __shfl_up_sync(FULL, cL, 1) >> 24;   // column q-1 of lane 0
            xP = (lUp << 4) | cL;
            yP = (((cL << 8) | lNb) << 4) | cL;
        }
        bool active = true;
        if (GENERAL) {
            const int lo = (ln.y0 == 0) ? 0 : (ln.y0 - K + k);
            const int hi = min(ln.ny, ln.y1 + K - k - 1);
            active = (r >= lo && r < hi);
        }
        if (active) {
            const int64_t n = n0 + k;
            const float yR = __shfl_down_sync(FULL, p.Y[k][0], 1);
            const bool tf = GENERAL && (r == a.s.js);
            const float hinc = tf ? tab(a.s.hinc, n, a.s) : 0.f;
            const int pe = GENERAL ? pml_e_index(r, ln.ny, ln.P) : -1;
            if (GENERAL && pe >= 0 && index_ok(pe < 2 * ln.P, kSitePsiRow, a.s.dbg)) {
                const float b = a.s.pml_e[pe], c = a.s.pml_e[2 * ln.P + pe];
                const float ik = a.s.pml_e[4 * ln.P + pe];
                float psi[4];
                if (k == 0) {
                    if (ln.col_ok) ld4(a.psiE_in + (size_t)pe * a.s.pitch + ln.gx, psi);
                    else psi[0] = psi[1] = psi[2] = psi[3] = 0.f;
                }
                else {
                    const float4 v = ringE[(r % K) * 32];
                    psi[0] = v.x; psi[1] = v.y; psi[2] = v.z; psi[3] = v.w;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 cc = POL ? make_float2(1.0f, S) : coef_s<V>(ln, cL, q);
                    const float dhy = __fsub_rn(q < 3 ? p.Y[k][q + 1] : yR, p.Y[k][q]);
                    float dhx = __fsub_rn(fX[q], p.X[k][q]);
                    if (tf) dhx = __fsub_rn(dhx, hinc);
                    psi[q] = psi_new(b, c, psi[q], dhx);
                    if (V == 4 || V == 6) cu[q] = __fadd_rn(dhy, __fmaf_rn(dhx, ik, psi[q]));
                    oE[q] = ez_new_pml(cc.x, cc.y, p.E[k][q], dhy, dhx, ik, psi[q]);
                }
                if (k == K - 1) {
                    if (ln.own && r >= ln.y0 && r < ln.y1)
                        st4(a.psiE_out + (size_t)pe * a.s.pitch + ln.gx, psi);
                } else {
                    ringE[(r % K) * 32] = make_float4(psi[0], psi[1], psi[2], psi[3]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 cc = POL ? make_float2(1.0f, S) : coef_s<V>(ln, cL, q);
                    const float dhy = __fsub_rn(q < 3 ? p.Y[k][q + 1] : yR, p.Y[k][q]);
                    float dhx = __fsub_rn(fX[q], p.X[k][q]);
                    if (tf) dhx = __fsub_rn(dhx, hinc);
                    if (V == 4 || V == 6) cu[q] = __fadd_rn(dhy, dhx);
                    oE[q] = ez_new(cc.x, cc.y, p.E[k][q], dhy, dhx);
                }
            }
            if (!GENERAL || r > 0) {
                const float einc = tf ? tab(a.s.einc, n, a.s) : 0.f;
                const int ph = GENERAL ? pml_h_index(r, ln.ny, ln.P) : -1;
                if (GENERAL && ph >= 0 && index_ok(ph < 2 * ln.P, kSitePsiRow, a.s.dbg)) {
                    const float b = a.s.pml_h[ph], c = a.s.pml_h[2 * ln.P + ph];
                    const float ik = a.s.pml_h[4 * ln.P + ph];
                    float psi[4];
                    if (k == 0) {
                        if (ln.col_ok) ld4(a.psiH_in + (size_t)ph * a.s.pitch + ln.gx, psi);
                        else psi[0] = psi[1] = psi[2] = psi[3] = 0.f;
                    }
                    else {
                        const float4 v = ringH[(r % K) * 32];
                        psi[0] = v.x; psi[1] = v.y; psi[2] = v.z; psi[3] = v.w;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float d = __fsub_rn(oE[q], p.E[k + 1][q]);
                        if (tf) d = __fsub_rn(d, einc);
                        psi[q] = psi_new(b, c, psi[q], d);
                        if (POL == 1) {
                            const float2 cx = ln.coef[(xP >> (8 * q)) & 0xffu];
                            oX[q] = e_edge_new_pml(cx.x, cx.y, p.X[k][q], d, ik, psi[q]);
                        } else {
                            oX[q] = h_new_pml(p.X[k][q], S, d, ik, psi[q]);
                        }
                    }
                    if (k == K - 1) {
                        if (ln.own && r >= ln.y0 && r < ln.y1)
                            st4(a.psiH_out + (size_t)ph * a.s.pitch + ln.gx, psi);
                    } else {
                        ringH[(r % K) * 32] = make_float4(psi[0], psi[1], psi[2], psi[3]);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float d = __fsub_rn(oE[q], p.E[k + 1][q]);
                        if (tf) d = __fsub_rn(d, einc);
                        if (POL == 1) {
                            const float2 cx = ln.coef[(xP >> (8 * q)) & 0xffu];
                            oX[q] = e_edge_new(cx.x, cx.y, p.X[k][q], d);
                        } else {
                            oX[q] = h_new(p.X[k][q], S, d);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) oX[q] = p.X[k][q];
            }
            const float eL = __shfl_up_sync(FULL, oE[3], 1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float dy = __fsub_rn(oE[q], q > 0 ? oE[q - 1] : eL);
                if (POL == 1) {
                    const float2 cy = ln.coef[(yP >> (8 * q)) & 0xffu];
                    oY[q] = e_edge_new(cy.x, cy.y, p.Y[k][q], dy);
                } else {
                    oY[q] = h_new(p.Y[k][q], S, dy);
                }
            }
            if ((V == 4 || V == 6) && ln.own && r >= ln.y0 && r < ln.y1 &&
                index_ok(r >= 0 && r < ln.ny && ln.col_ok, kSiteTape, a.s.dbg)) {
                // code shapes 4, 6: step n0+k's gradient factors of this row
                // (Ez before the update and the factor of cb)
                float* t = a.tape[k] + (size_t)r * a.s.pitch + ln.gx;
                const float eo[4] = {p.E[k][0], p.E[k][1], p.E[k][2], p.E[k][3]};
                st4(t, eo);
                st4(t + a.tape_f, cu);
            }
            if (GENERAL && ln.own && index_ok(ln.col_ok, kSiteDft, a.s.dbg)) {
                if (ln.own_r && r == a.s.jr) {
                    const double2 ph = tab(a.s.phE, n, a.s);
#pragma unroll
                    for (int q = 0; q < 4; ++q) dft_add(&a.s.dft[ln.gx + q], oE[q], ph);
                }
                if (ln.own_r && r == a.s.jr + 1) {
                    const double2 ph = tab(a.s.phH, n, a.s);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dft_add(&a.s.dft[ln.nx + ln.gx + q], hx_avg(p.X[k + 1][q], oX[q]), ph);
                }
                if (ln.own_t && r == a.s.jt) {
                    const double2 ph = tab(a.s.phE, n, a.s);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dft_add(&a.s.dft[2 * ln.nx + ln.gx + q], oE[q], ph);
                }
                if (ln.own_t && r == a.s.jt + 1) {
                    const double2 ph = tab(a.s.phH, n, a.s);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dft_add(&a.s.dft[3 * ln.nx + ln.gx + q], hx_avg(p.X[k + 1][q], oX[q]),
                                ph);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) { oE[q] = 0.f; oX[q] = 0.f; oY[q] = 0.f; }
        }
        // level k now waits at row r+1; the new level-(k+1) row r flows up
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            p.E[k][q] = fE[q]; p.X[k][q] = fX[q]; p.Y[k][q] = fY[q];
            fE[q] = oE[q]; fX[q] = oX[q]; fY[q] = oY[q];
        }
        p.L[k] = fL;
        fL = cL;
        if (POL == 1 && kPairShape<V>) {
            const uint32_t cY = p.LY[k];
            p.LY[k] = fLY;
            fLY = cY;
        }
        if (POL == 1 && k == K - 1) p.L[K] = cL;
    }
}

// One warp task: strip `task % n_strips` of segment `task / n_strips`.
// Code shapes V: 0 one row per loop trip with a one-row register prefetch;
// 1 two rows per loop trip on plain stretches; 2 level-0 rows streamed
// through a shared-memory ring filled kRing rows ahead by cp.async, two rows
// per loop trip on lean stretches; 3 the ring with one row per trip (built
// under a register cap, see k_blocked_cap); 4 the ring, one row per trip,
// that also stores, for each step n of the launch and each owned row, the
// two factors of the adjoint's gradient sums, Ez^{n-1/2} and the factor of
// cb in the Ez update (the curl with its CPML and TF/SF terms), into
// BlockedArgs::tape, for the adjoint's recompute;
// 5 (at most 16 labels) shape 2 with paired FP32 instructions on the lean
// path: for S with the label-pair coefficient table (advance_lean_pair),
// for P on the centre update and the edge differences along s
// (advance_lean_pair_p); 6 (S, at most 16 labels) shape 4 with the
// label-pair table, the paired lean path and two lean rows per trip (the
// adjoint's recompute). In shapes 5 and 6 the two lean rows of a loop trip
// run skewed by one level (advance_lean_pair2), which exposes two
// independent dependency chains.
template <int K, int V, int POL>
__device__ __forceinline__ void blocked_task(const BlockedArgs& a, const float4* s_tab,
                                             const int task, const int64_t n0) {
    constexpr int H = ((K + 3) / 4) * 4;
    const int lane = threadIdx.x & 31;
    const int strip = task % a.n_strips;
    const int seg = task / a.n_strips;
    Lane ln;
    ln.coef = reinterpret_cast<const float2*>(s_tab);
    ln.pair = s_tab;
    ln.y0 = a.seg_y0[seg];
    ln.y1 = a.seg_y0[seg + 1];
    ln.nx = a.s.nx; ln.ny = a.s.ny; ln.P = a.s.P; ln.S = a.s.S;
    const size_t pitch = (size_t)a.s.pitch;
    const size_t lpitch = (size_t)a.s.lpitch;
    const int xl = 4 * lane;                        // local column of the lane
    const int xg_pre = strip * a.w_int - H + xl;    // global column before wrapping
    ln.gx = ((xg_pre % ln.nx) + ln.nx) % ln.nx;     // nx % 4 == 0: 4 columns stay contiguous
    ln.own = (xl >= H) && (xl < H + a.w_int) && (xg_pre < ln.nx);
    ln.col_ok = index_ok(ln.gx >= 0 && ln.gx + 4 <= ln.nx && ln.gx % 4 == 0, kSiteRingColumn,
                         a.s.dbg);
    ln.own = ln.own && ln.col_ok;      // a lane with bad columns stores nothing
    ln.own_r = (a.s.jr >= ln.y0) && (a.s.jr < ln.y1);
    ln.own_t = (a.s.jt >= ln.y0) && (a.s.jt < ln.y1);
    // CPML carries between levels: psi of a row is written by level k and
    // read by level k+1 one iteration later, so K rows are in flight; a
    // lane-private shared-memory ring indexed by row mod K holds them.
    __shared__ float4 s_psi[2][K][32];
    float4* ringE = &s_psi[0][0][lane];
    float4* ringH = &s_psi[1][0][lane];

    Pipe<K> p;
#pragma unroll
    for (int k = 0; k <= K; ++k) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            p.E[k][q] = 0.f; p.X[k][q] = 0.f;
            if (k < K) p.Y[k][q] = 0.f;
        }
        p.L[k] = 0u;
        if (k < K) p.LY[k] = 0u;
    }

    const int y0 = ln.y0, y1 = ln.y1, ny = ln.ny, P = ln.P;
    const int t_begin = (y0 == 0) ? 0 : (y0 - K);
    const int t_end = y1 + K;
    // Iterations whose rows t-K .. t-1 hold no CPML, source or monitor row
    // take the lean path. That includes the first iterations of a segment,
    // where some levels are still outside their valid row range: the lean
    // path computes values there that no stored row ever depends on (each
    // level's valid range shrinks by one row per step, exactly the reach of
    // a step), and it has no other side effect.
    const int fast_lo = max(K + 1, P + K);
    const int fast_hi = ny - P + 1;
    const int sp[5] = {a.s.js, a.s.jr, a.s.jr + 1, a.s.jt, a.s.jt + 1};
    auto is_fast = [&](int t) {
        bool f = (t >= fast_lo) && (t < fast_hi);
#pragma unroll
        for (int s = 0; s < 5; ++s) f = f && ((unsigned)(t - sp[s] - 1) >= (unsigned)K);
        return f;
    };

    auto finish = [&](const int t, V4& fE, V4& fX, V4& fY) {
        const int ro = t - K;
        if (ln.own && ro >= y0 && ro < y1 &&
            index_ok(ro >= 0 && ro < ny, kSiteStoreRow, a.s.dbg)) {
            const size_t o = (size_t)ro * pitch + ln.gx;
            st4(a.ez_out + o, fE);
            st4(a.hx_out + o, fX);
            st4(a.hy_out + o, fY);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) { p.E[K][q] = fE[q]; p.X[K][q] = fX[q]; }
    };

    if (V >= 2) {
        uint32_t prevL = 0u;   // P, code shape 5: label word of the previous level-0 row
        __shared__ float4 ring[kRing][3][32];
        __shared__ uint32_t ring_l[kRing][32];
        auto issue = [&](const int row, const int slot) {
            const bool ok = row >= 0 && row < ny && ln.col_ok;
            const size_t o = (size_t)(ok ? row : 0) * pitch + ln.gx;
            const int nb = ok ? 16 : 0;
            cp_async16(&ring[slot][0][lane], a.ez_in + o, nb);
            cp_async16(&ring[slot][1][lane], a.hx_in + o, nb);
            cp_async16(&ring[slot][2][lane], a.hy_in + o, nb);
            cp_async4(&ring_l[slot][lane], a.s.labels + (size_t)(ok ? row : 0) * lpitch + ln.gx,
                      ok ? 4 : 0);
            cp_async_commit();
        };
#pragma unroll
        for (int d = 0; d < kRing; ++d) issue(t_begin + d, d);
        int slot = 0;
        // the level-0 row of ring slot `sl` as pipeline input
        auto take = [&](const int sl, V4& fE, V4& fX, V4& fY, uint32_t& fL, uint32_t& fLY) {
            const float4 e4 = ring[sl][0][lane], x4 = ring[sl][1][lane], y4 = ring[sl][2][lane];
            fL = ring_l[sl][lane];
            // every label must index the coefficient table (debug builds)
            index_ok(((fL & 0xffu) < (unsigned)a.s.n_labels) &&
                         (((fL >> 8) & 0xffu) < (unsigned)a.s.n_labels) &&
                         (((fL >> 16) & 0xffu) < (unsigned)a.s.n_labels) &&
                         ((fL >> 24) < (unsigned)a.s.n_labels),
                     kSiteLabel, a.s.dbg);
            if (kPairShape<V> && POL == 0) fL = pair_offsets(fL);
            // P, code shape 5: the row's edge label pairs, formed once here
            // (top edges pair rows t-1 and t, left edges columns q-1 and q)
            fLY = 0u;
            if (kPairShape<V> && POL == 1) {
                const uint32_t raw = fL;
                const uint32_t lNb = __shfl_up_sync(FULL, raw, 1) >> 24;   // column q-1 of lane 0
                fLY = (((raw << 8) | lNb) << 4) | raw;
                fL = (prevL << 4) | raw;
                prevL = raw;
            }
            fE.a = make_float2(e4.x, e4.y); fE.b = make_float2(e4.z, e4.w);
            fX.a = make_float2(x4.x, x4.y); fX.b = make_float2(x4.z, x4.w);
            fY.a = make_float2(y4.x, y4.y); fY.b = make_float2(y4.z, y4.w);
        };
        // two lean rows t, t+1 (code shape 5), skewed by one level
        auto row2 = [&](const int t) {
            cp_async_wait<kRing - 2>();
            V4 fE0, fX0, fY0, fE1, fX1, fY1;
            uint32_t fL0, fLY0, fL1, fLY1;
            const int s1 = (slot + 1 == kRing) ? 0 : slot + 1;
            take(slot, fE0, fX0, fY0, fL0, fLY0);
            take(s1, fE1, fX1, fY1, fL1, fLY1);
            issue(t + kRing, slot);
            issue(t + 1 + kRing, s1);
            slot = (s1 + 1 == kRing) ? 0 : s1 + 1;
            advance_lean_pair2<K, V, POL>(p, fE0, fX0, fY0, fL0, fLY0, fE1, fX1, fY1, fL1, fLY1,
                                       ln, a, t, [&]() { finish(t, fE0, fX0, fY0); });
            finish(t + 1, fE1, fX1, fY1);
        };
        auto row = [&](const int t, const bool fast) {
            cp_async_wait<kRing - 1>();
            V4 fE, fX, fY;
            uint32_t fL, fLY;
            take(slot, fE, fX, fY, fL, fLY);
            issue(t + kRing, slot);
            slot = (slot + 1 == kRing) ? 0 : slot + 1;
            if (fast) advance<K, false, POL, V>(p, fE, fX, fY, fL, fLY, t, a, ln, ringE, ringH, n0);
            else advance<K, true, POL, V>(p, fE, fX, fY, fL, fLY, t, a, ln, ringE, ringH, n0);
            finish(t, fE, fX, fY);
        };
        // Two lean rows per loop trip: every pipeline register is replaced
        // each row while its old value is still being read, so a one-row
        // loop copies the new values back at the end of each trip; over two
        // rows the two register sets alternate and the copies disappear.
#pragma unroll 1
        for (int t = t_begin; t < t_end;) {
            if (kPairShape<V> && t + 1 < t_end && is_fast(t) && is_fast(t + 1)) {
                row2(t);
                t += 2;
            } else if ((V == 2 || V == 5) && t + 1 < t_end && is_fast(t) && is_fast(t + 1)) {
                row(t, true);
                row(t + 1, true);
                t += 2;
            } else {
                row(t, is_fast(t));
                t += 1;
            }
        }
        cp_async_wait<0>();
        return;
    }

    // software pipeline: row t+1 is fetched while row t is processed
    float nE[4], nX[4], nY[4];
    uint32_t nL = 0u;
    if (ln.col_ok && index_ok(t_begin >= 0 && t_begin < ny, kSiteStoreRow, a.s.dbg)) {
        const size_t o = (size_t)t_begin * pitch + ln.gx;
        ld4(a.ez_in + o, nE);
        ld4(a.hx_in + o, nX);
        ld4(a.hy_in + o, nY);
        nL = __ldg(reinterpret_cast<const uint32_t*>(a.s.labels + (size_t)t_begin * lpitch + ln.gx));
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) { nE[q] = 0.f; nX[q] = 0.f; nY[q] = 0.f; }
    }
    auto iteration = [&](const int t, const bool fast) {
        V4 fE, fX, fY;
        uint32_t fL = nL, fLY = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) { fE[q] = nE[q]; fX[q] = nX[q]; fY[q] = nY[q]; }
        if (t + 1 < ny && ln.col_ok) {
            const size_t o = (size_t)(t + 1) * pitch + ln.gx;
            ld4(a.ez_in + o, nE);
            ld4(a.hx_in + o, nX);
            ld4(a.hy_in + o, nY);
            nL = __ldg(reinterpret_cast<const uint32_t*>(a.s.labels + (size_t)(t + 1) * lpitch + ln.gx));
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) { nE[q] = 0.f; nX[q] = 0.f; nY[q] = 0.f; }
            nL = 0u;
        }
        if (fast) advance<K, false, POL, V>(p, fE, fX, fY, fL, fLY, t, a, ln, ringE, ringH, n0);
        else advance<K, true, POL, V>(p, fE, fX, fY, fL, fLY, t, a, ln, ringE, ringH, n0);
        finish(t, fE, fX, fY);
    };
    int t = t_begin;
#pragma unroll 1
    while (t < t_end) {
        if (V == 1 && t + 1 < t_end && is_fast(t) && is_fast(t + 1)) {
            iteration(t, true);
            iteration(t + 1, true);
            t += 2;
        } else {
            if (is_fast(t)) iteration(t, true);
            else iteration(t, false);
            t += 1;
        }
    }
}

// Coefficients of a block in shared memory: the per-label (S) or per-label-
// pair (P) float2 table, or for code shape 5 the S label-pair table of
// float4 entries (ca[b0], ca[b1], cb[b0], cb[b1]) at index b0 | b1 << 4,
// built from the per-label table (labels < 16).
template <int V, int POL>
__device__ __forceinline__ void load_coef_table(const StepArgs& s, float4* s_tab) {
    if (kPairShape<V> && POL == 0) {
        const int last = s.n_labels - 1;
        for (int t = threadIdx.x; t < 256; t += 32) {
            const float2 c0 = s.coef[min(t & 15, last)], c1 = s.coef[min(t >> 4, last)];
            s_tab[t] = make_float4(c0.x, c1.x, c0.y, c1.y);
        }
    } else {
        float2* s_coef = reinterpret_cast<float2*>(s_tab);
        const int n_coef = POL ? 256 : s.n_labels;
        for (int t = threadIdx.x; t < n_coef; t += 32) s_coef[t] = s.coef[t];
    }
    __syncwarp();
}

template <int K, int V, int POL>
__device__ __forceinline__ void blocked_kernel_body(const BlockedArgs& a, const int64_t n0) {
    __shared__ float4 s_tab[(kPairShape<V> && POL == 0) ? 256 : 128];
    load_coef_table<V, POL>(a.s, s_tab);
    if ((int)blockIdx.x >= a.n_tasks) return;       // one warp per block and task
    blocked_task<K, V, POL>(a, s_tab, blockIdx.x, n0);
}

template <int K, int V, int POL>
__global__ void __launch_bounds__(32) k_blocked(const BlockedArgs a, const int64_t n0) {
    blocked_kernel_body<K, V, POL>(a, n0);
}

// Code shape 3: the ring with one row per loop trip, compiled under a
// 224-register cap (8 one-warp blocks per SM). The two-row trip of shape 2
// does not fit under the cap without spills; shape 3 stays available as an
// option (and as the one-row form of the same pipeline).
template <int K, int POL>
__global__ void __maxnreg__(224) k_blocked_cap(const BlockedArgs a,
                                                                     const int64_t n0) {
    blocked_kernel_body<K, 3, POL>(a, n0);
}

template <int K, int V, int POL>
__device__ __forceinline__ void blocked_batch_body(const BatchArgs& b, const int step_off,
                                                   const int parity) {
    __shared__ float4 s_tab[(kPairShape<V> && POL == 0) ? 256 : 128];
    __shared__ __align__(16) unsigned char s_raw[sizeof(BlockedArgs)];
    const int task = blockIdx.x;
    if (task >= b.n_tasks) return;
    const int sim = b.task_sim[task];
    const BlockedArgs* src = b.sims + (size_t)parity * b.n_sims + sim;
    const int* w = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(s_raw);
    for (int q = threadIdx.x; q < (int)(sizeof(BlockedArgs) / sizeof(int)); q += 32) d[q] = w[q];
    __syncwarp();
    const BlockedArgs& a = *reinterpret_cast<const BlockedArgs*>(s_raw);
    load_coef_table<V, POL>(a.s, s_tab);
    const int64_t n0 = a.n_base + *b.step_base + step_off;
    blocked_task<K, V, POL>(a, s_tab, task - b.first_task[sim], n0);
}

// Many independent simulations in one launch: the grid covers the union of
// their warp tasks. Each block finds its simulation, copies that
// simulation's arguments (ping-pong orientation `parity`) to shared memory
// and runs the same task body. The absolute step of the launch is
// n_base(sim) + *step_base + step_off, so a captured chunk of launches can be
// replayed with a new *step_base.
template <int K, int V, int POL>
__global__ void __launch_bounds__(32) k_blocked_batch(const BatchArgs b, const int step_off,
                                                      const int parity) {
    blocked_batch_body<K, V, POL>(b, step_off, parity);
}

template <int K, int POL>
__global__ void __maxnreg__(224) k_blocked_batch_cap(const BatchArgs b,
                                                                           const int step_off,
                                                                           const int parity) {
    blocked_batch_body<K, 3, POL>(b, step_off, parity);
}

template <typename F>
inline int occupancy_of(F kernel) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 32, 0) != cudaSuccess) return 0;
    return b;
}

// Per-translation-unit entry points (one per instantiated family).
int blocked_occupancy_s(int K, int variant);
int blocked_occupancy_p(int K, int variant);
bool launch_blocked_s(const BlockedArgs& a, int K, int variant, int64_t n0, cudaStream_t st);
bool launch_blocked_p(const BlockedArgs& a, int K, int variant, int64_t n0, cudaStream_t st);
bool launch_blocked_batch_s(const BatchArgs& b, int K, int variant, int step_off, int parity,
                            cudaStream_t st);
bool launch_blocked_batch_p(const BatchArgs& b, int K, int variant, int step_off, int parity,
                            cudaStream_t st);

#define FDTD_BLOCKED_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8)

}  // namespace fdtd
