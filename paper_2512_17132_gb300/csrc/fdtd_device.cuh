// Device-side update arithmetic shared by every field-update kernel of the
// library, so that the per-half-step kernels, the temporally blocked kernel
// and the empty-domain column kernel round identically (explicit _rn
// intrinsics keep the compiler from contracting them differently).
//
// Units: Ez in V/m, H stored as eta0*H (V/m). With S = c0 dt/dx the TMz
// updates of Sec. 2.3 become
//   Ez <- ca Ez + cb [ (Hy[i+1]-Hy[i]) + (Hx[j+1]-Hx[j]) ]
//   Hx <- Hx + S (Ez[j] - Ez[j-1]),   Hy <- Hy + S (Ez[i] - Ez[i-1])
// with ca = (1-b)/(1+b), cb = S/(eps_r (1+b)), b = sigma dt/(2 eps0 eps_r).
// In CPML rows the s-derivative d is replaced by d/kappa + psi with
// psi <- b_pml psi + c_pml d (Roden-Gedney recursive convolution).
//
// P polarisation (TEz) runs on the same three buffers with the variables
// F = eta0 Hz (centre), X = -Ex (top edge), Y = -Ey (left edge). In them the
// TEz updates of Sec. 2.3 take the TMz form with the loss coefficients moved
// from the centre to the edges:
//   F <- F + S [ (Y[i+1]-Y[i]) + (X[j+1]-X[j]) ]
//   X <- ce X + cb (F[j] - F[j-1]),   Y <- ce Y + cb (F[i] - F[i-1])
// where (ce, cb) of an edge come from the mean eps_r and sigma of the two
// cells it separates, and the incident pair, CPML, DFT and flux are those of
// the TMz run (the TMz/TEz duality of the air lattice).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fdtd {

__device__ __forceinline__ float ez_new(float ca, float cb, float e, float dhy, float dhx) {
    return __fmaf_rn(cb, __fadd_rn(dhy, dhx), __fmul_rn(ca, e));
}

__device__ __forceinline__ float ez_new_pml(float ca, float cb, float e, float dhy,
                                            float dhx, float ik, float psi) {
    return __fmaf_rn(cb, __fadd_rn(dhy, __fmaf_rn(dhx, ik, psi)), __fmul_rn(ca, e));
}

__device__ __forceinline__ float psi_new(float b, float c, float psi, float d) {
    return __fmaf_rn(b, psi, __fmul_rn(c, d));
}

__device__ __forceinline__ float h_new(float h, float S, float d) {
    return __fmaf_rn(S, d, h);
}

__device__ __forceinline__ float h_new_pml(float h, float S, float d, float ik, float psi) {
    return __fmaf_rn(S, __fmaf_rn(d, ik, psi), h);
}

// Lossy edge update of P polarisation: ce X + cb d, and its CPML form.
__device__ __forceinline__ float e_edge_new(float ce, float cb, float x, float d) {
    return __fmaf_rn(cb, d, __fmul_rn(ce, x));
}

__device__ __forceinline__ float e_edge_new_pml(float ce, float cb, float x, float d, float ik,
                                                float psi) {
    return __fmaf_rn(cb, __fmaf_rn(d, ik, psi), __fmul_rn(ce, x));
}

// Index of the edge coefficient pair of two labels (< 16 each) in the
// 256-entry table of a P-polarised handle.
__device__ __forceinline__ int pair_index(unsigned la, unsigned lb) { return (int)((la << 4) | lb); }

// Row-averaged Hx at a monitor row: edges row and row+1.
__device__ __forceinline__ float hx_avg(float a, float b) {
    return __fmul_rn(0.5f, __fadd_rn(a, b));
}

__device__ __forceinline__ void dft_add(double2* acc, float v, double2 ph) {
    double2 a = *acc;
    a.x = fma((double)v, ph.x, a.x);
    a.y = fma((double)v, ph.y, a.y);
    *acc = a;
}

// Index checks of debug builds. Built with FDTD_DEBUG_BOUNDS, the kernels
// test every global-memory index that is not in range by construction; a
// failed test sets the bit of its site in the handle's error word and the
// access is skipped (a load reads 0), so the kernel finishes and the host
// reports FDTD_EBOUNDS. Release builds compile the tests away.
enum CheckSite : unsigned {
    kSiteRingColumn = 0,   // blocked: lane columns of a level-0 row load
    kSiteStoreRow = 1,     // blocked: row and columns of a stored row
    kSitePsiRow = 2,       // CPML carry row index
    kSiteTable = 3,        // incident / phase table entry (step index)
    kSiteDft = 4,          // monitor accumulator column
    kSiteLabel = 5,        // label value against the coefficient table
    kSiteTape = 6,         // adjoint tape row
    kSiteTask = 7,         // warp task / segment index
};

__device__ __forceinline__ bool index_ok(bool ok, unsigned site, unsigned* err) {
#ifdef FDTD_DEBUG_BOUNDS
    if (!ok && err) atomicOr(err, 1u << site);
    return ok;
#else
    (void)site; (void)err;
    return true;
#endif
}

// Arguments common to the field-update kernels.
struct StepArgs {
    int nx, ny;
    int pitch;            // floats per field row (multiple of 32)
    int lpitch;           // bytes per label row (multiple of 16)
    int P;                // CPML rows per side
    int js, jr, jt;       // TF/SF row, monitor rows
    int n_labels;
    int pol;              // 0: S (TMz), 1: P (TEz)
    float S;              // Courant number c0 dt / dx
    const uint8_t* labels;
    const float2* coef;   // S: (ca, cb) per label; P: (ce, cb) per label pair (pair_index)
    const float2* cellcoef;  // (ca, cb) per cell (pitch floats2 per row) or null
    const float* pml_e;   // [3][2P]: b, c, 1/kappa for Ez rows (top 0..P-1, then bottom)
    const float* pml_h;   // [3][2P]: same for Hx rows
    const float* hinc;    // incident eta0*Hx at edge tfsf_row, per absolute step
    const float* einc;    // incident Ez at cell tfsf_row, per absolute step
    const double2* phE;   // e^{i w0 (n+1/2) dt}
    const double2* phH;   // e^{i w0 (n+1) dt}
    double2* dft;         // [4][nx]: Ez(jr), Hx(jr), Ez(jt), Hx(jt)
    int64_t n_tab;        // table entries valid on the device (debug index checks)
    int n_coef;           // entries of coef (debug index checks)
    unsigned* dbg;        // error word of the debug index checks (null: none)
};

// Table entry n of the incident / phase tables of n_tab entries; debug
// builds check n.
template <typename T>
__device__ __forceinline__ T tab_n(const T* t, int64_t n, int64_t n_tab, unsigned* dbg) {
    return index_ok(n >= 0 && n < n_tab, kSiteTable, dbg) ? t[n] : T{};
}
template <typename T>
__device__ __forceinline__ T tab(const T* t, int64_t n, const StepArgs& s) {
    return tab_n(t, n, s.n_tab, s.dbg);
}

// Coefficients of a label (S: per label, P: per label pair); debug builds
// check the index against the table.
__device__ __forceinline__ float2 coef_at(const StepArgs& s, int idx) {
    return index_ok(idx >= 0 && idx < s.n_coef, kSiteLabel, s.dbg) ? s.coef[idx]
                                                                    : make_float2(0.f, 0.f);
}

// Index of a CPML row within the [2P] tables and psi arrays, or -1.
__device__ __forceinline__ int pml_e_index(int j, int ny, int P) {
    return (j < P) ? j : ((j >= ny - P) ? (P + j - (ny - P)) : -1);
}
__device__ __forceinline__ int pml_h_index(int j, int ny, int P) {
    return (j < P) ? j : ((j >= ny - P) ? (P + j - (ny - P)) : -1);
}

}  // namespace fdtd
