/* Plain FP64 time loop of the 2D TMz Yee scheme (Sec. 2.3 to 2.6), in C.
 *
 * TEST INFRASTRUCTURE. This is the same discrete system as the numpy oracle
 * (oracle/fdtd_tmz.py), written as plain loops over rows j and columns i so
 * that full-size grids (tens of millions of cells, tens of thousands of
 * steps) finish on the host cores in tens of minutes instead of many hours.
 * Each update equation is one loop nest; the arithmetic of every cell is the
 * numpy oracle's, operation for operation (same operands, same order, no
 * fused multiply-add: build with -ffp-contract=off), so the two oracles agree
 * bit for bit. Rows are shared among OpenMP threads; no blocking, fusion of
 * the E and H passes or reordering of the time loop.
 *
 * Conventions (rows counted downward, s = -y, periodic columns):
 *   Ez[j][i]  cell centre, times n+1/2;  Hx[j][i] top edge, Hy[j][i] left
 *   edge, times n.  Hx[0] and the virtual Hx[ny] are 0.
 *   Ez <- ce Ez + ce_curl curl H,  curl H = (Hy[i+1]-Hy[i] + Hx[j+1]-Hx[j])/dx
 *   Hx[j] += ch (Ez[j]-Ez[j-1])/dx (j >= 1), Hy[i] += ch (Ez[i]-Ez[i-1])/dx
 *   CFS-CPML rows: the s-difference d becomes d/kappa + psi, psi <- b psi + c d
 *   TF/SF (Sec. 2.5): cell js sees Hx[js] + h_inc, edge js sees Ez[js] - e_inc
 *   running DFTs (Sec. 2.6): Ez rows jr, jt at n+1/2 and the mean of the two
 *   Hx edges of each row at n+1, each times its phase factor.
 *
 * The caller (oracle/fdtd_tmz_c.py) passes the per-cell coefficients, the
 * CPML profiles, the incident samples and the DFT phases, all computed by
 * the numpy oracle's own functions.
 */
#include <stddef.h>
#include <stdint.h>

typedef struct {
    int32_t nx, ny;
    double dx;
    double ch_curl;        /* dt / mu0 */
    int32_t js, tfsf;      /* TF/SF row and whether the source is on */
    int32_t jr, jt;        /* monitor rows */
    int32_t threads;
} tmz_loop_args;

/* pml_e_idx[j]: index of Ez row j among the CPML rows (-1 outside);
 * pml_h_idx[j]: the same for Hx row j. b, c, kappa are per CPML row.
 * psi_e, psi_h: (number of CPML rows) x nx.
 * h_inc, e_inc, ph_e, ph_h: per step of this call (phases as re, im pairs).
 * dft: e_r, h_r, e_t, h_t, each nx complex numbers as re, im pairs. */
int tmz_loop_run(const tmz_loop_args *a, int64_t steps,
                 double *ez, double *hx, double *hy,
                 const double *ce, const double *ce_curl,
                 const int32_t *pml_e_idx, const double *eb, const double *ec,
                 const double *ek, double *psi_e,
                 const int32_t *pml_h_idx, const double *hb, const double *hc,
                 const double *hk, double *psi_h,
                 const double *h_inc, const double *e_inc,
                 const double *ph_e, const double *ph_h, double *dft)
{
    const int64_t nx = a->nx, ny = a->ny;
    const double dx = a->dx, ch = a->ch_curl;
    double *dft_er = dft, *dft_hr = dft + 2 * nx, *dft_et = dft + 4 * nx, *dft_ht = dft + 6 * nx;
    if (nx < 1 || ny < 2 || a->jr < 0 || a->jt < 0 || a->jr + 1 >= ny || a->jt + 1 >= ny)
        return -1;
    if (a->tfsf && (a->js < 1 || a->js >= ny))
        return -1;

    for (int64_t n = 0; n < steps; ++n) {
        const double hin = h_inc[n], ein = e_inc[n];

        /* Ez^{n-1/2} -> Ez^{n+1/2} */
#pragma omp parallel for schedule(static) num_threads(a->threads)
        for (int64_t j = 0; j < ny; ++j) {
            double *ezr = ez + j * nx;
            const double *hxr = hx + j * nx;
            const double *hyr = hy + j * nx;
            const double *cer = ce + j * nx, *ccr = ce_curl + j * nx;
            const int32_t p = pml_e_idx[j];
            for (int64_t i = 0; i < nx; ++i) {
                const double hx_below = (j + 1 < ny) ? hxr[nx + i] : 0.0;
                double d_hx = hx_below - hxr[i];
                if (a->tfsf && j == a->js)
                    d_hx = d_hx - hin;
                const int64_t ip = (i + 1 == nx) ? 0 : i + 1;
                const double d_hy = hyr[ip] - hyr[i];
                double curl;
                if (p >= 0) {
                    double *ps = psi_e + (int64_t)p * nx + i;
                    *ps = *ps * eb[p];
                    *ps = *ps + ec[p] * d_hx / dx;
                    curl = d_hy / dx + d_hx / (ek[p] * dx) + *ps;
                } else {
                    curl = (d_hy + d_hx) / dx;
                }
                ezr[i] = cer[i] * ezr[i] + ccr[i] * curl;
            }
        }
        {
            const double c = ph_e[2 * n], s = ph_e[2 * n + 1];
            const double *er = ez + (int64_t)a->jr * nx, *et = ez + (int64_t)a->jt * nx;
            for (int64_t i = 0; i < nx; ++i) {
                dft_er[2 * i] += er[i] * c;
                dft_er[2 * i + 1] += er[i] * s;
                dft_et[2 * i] += et[i] * c;
                dft_et[2 * i + 1] += et[i] * s;
            }
        }

        /* H^n -> H^{n+1} */
#pragma omp parallel for schedule(static) num_threads(a->threads)
        for (int64_t j = 0; j < ny; ++j) {
            const double *ezr = ez + j * nx;
            double *hxr = hx + j * nx;
            double *hyr = hy + j * nx;
            if (j >= 1) {
                const int32_t p = pml_h_idx[j];
                for (int64_t i = 0; i < nx; ++i) {
                    double d_ez = ezr[i] - ezr[i - nx];
                    if (a->tfsf && j == a->js)
                        d_ez = d_ez - ein;
                    double term;
                    if (p >= 0) {
                        double *ps = psi_h + (int64_t)p * nx + i;
                        *ps = *ps * hb[p];
                        *ps = *ps + hc[p] * d_ez / dx;
                        term = d_ez / (hk[p] * dx) + *ps;
                    } else {
                        term = d_ez / dx;
                    }
                    hxr[i] = hxr[i] + ch * term;
                }
            }
            for (int64_t i = 0; i < nx; ++i) {
                const int64_t im = (i == 0) ? nx - 1 : i - 1;
                const double d_ez_x = ezr[i] - ezr[im];
                hyr[i] = hyr[i] + ch * d_ez_x / dx;
            }
        }
        {
            const double c = ph_h[2 * n], s = ph_h[2 * n + 1];
            const double *r0 = hx + (int64_t)a->jr * nx, *t0 = hx + (int64_t)a->jt * nx;
            for (int64_t i = 0; i < nx; ++i) {
                const double hr = 0.5 * (r0[i] + r0[nx + i]);
                const double ht = 0.5 * (t0[i] + t0[nx + i]);
                dft_hr[2 * i] += hr * c;
                dft_hr[2 * i + 1] += hr * s;
                dft_ht[2 * i] += ht * c;
                dft_ht[2 * i + 1] += ht * s;
            }
        }
    }
    return 0;
}
