/* Plain FP64 time loop of the 2D TEz Yee scheme (Sec. 2.3 to 2.6), in C.
 *
 * TEST INFRASTRUCTURE. The same discrete system as the numpy oracle
 * (oracle/fdtd_tez.py, TEzOracle.step), written as plain loops over rows j
 * and columns i so that full-size P-polarised grids finish on the host
 * cores in tens of minutes. Each update equation is one loop nest; every
 * cell takes the numpy oracle's operations on the same operands in the same
 * order (build with -ffp-contract=off: no fused multiply-add), so the two
 * oracles agree bit for bit. Rows are shared among OpenMP threads; no
 * blocking, fusion of the H and E passes or reordering of the time loop.
 *
 * Conventions (rows counted downward, s = -y, periodic columns):
 *   Hz[j][i] cell centre, times n+1/2; Ex[j][i] top edge, Ey[j][i] left
 *   edge, times n. Ex[0] and the virtual Ex[ny] are 0.
 *   Hz <- Hz - ch curl E,  curl E = (Ey[i+1]-Ey[i] + Ex[j+1]-Ex[j]) / dx
 *   Ex[j] <- cex Ex[j] - cex_curl (Hz[j]-Hz[j-1]) / dx   (j >= 1)
 *   Ey[i] <- cey Ey[i] - cey_curl (Hz[i]-Hz[i-1]) / dx
 *   CFS-CPML rows: the s-difference d becomes d/kappa + psi, psi <- b psi + c d
 *   TF/SF (Sec. 2.5): cell js sees Ex[js] - e_inc, edge js sees Hz[js] - h_inc
 *   running DFTs (Sec. 2.6): Hz rows jr, jt at n+1/2 and the mean of the two
 *   Ex edges of each row at n+1, each times its phase factor.
 *
 * The caller (oracle/fdtd_tez_c.py) passes the per-edge coefficients, the
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
} tez_loop_args;

/* pml_c_idx[j]: index of Hz row j among the CPML centre rows (-1 outside);
 * pml_x_idx[j]: the same for Ex row j. b, c, kappa are per CPML row;
 * psi_c, psi_x: (number of CPML rows) x nx.
 * e_inc, h_inc, ph_h, ph_e: per step of this call (phases as re, im pairs).
 * dft: h_r, e_r, h_t, e_t, each nx complex numbers as re, im pairs. */
int tez_loop_run(const tez_loop_args *a, int64_t steps,
                 double *hz, double *ex, double *ey,
                 const double *cex, const double *cex_curl,
                 const double *cey, const double *cey_curl,
                 const int32_t *pml_c_idx, const double *cb, const double *cc,
                 const double *ck, double *psi_c,
                 const int32_t *pml_x_idx, const double *xb, const double *xc,
                 const double *xk, double *psi_x,
                 const double *e_inc, const double *h_inc,
                 const double *ph_h, const double *ph_e, double *dft)
{
    const int64_t nx = a->nx, ny = a->ny;
    const double dx = a->dx, ch = a->ch_curl;
    double *dft_hr = dft, *dft_er = dft + 2 * nx, *dft_ht = dft + 4 * nx, *dft_et = dft + 6 * nx;
    if (nx < 1 || ny < 2 || a->jr < 0 || a->jt < 0 || a->jr + 1 >= ny || a->jt + 1 >= ny)
        return -1;
    if (a->tfsf && (a->js < 1 || a->js >= ny))
        return -1;

    for (int64_t n = 0; n < steps; ++n) {
        const double ein = e_inc[n], hin = h_inc[n];

        /* Hz^{n-1/2} -> Hz^{n+1/2} */
#pragma omp parallel for schedule(static) num_threads(a->threads)
        for (int64_t j = 0; j < ny; ++j) {
            double *hzr = hz + j * nx;
            const double *exr = ex + j * nx;
            const double *eyr = ey + j * nx;
            const int32_t p = pml_c_idx[j];
            for (int64_t i = 0; i < nx; ++i) {
                const double ex_below = (j + 1 < ny) ? exr[nx + i] : 0.0;
                double d_ex = ex_below - exr[i];
                if (a->tfsf && j == a->js)
                    d_ex = d_ex - ein;
                const int64_t ip = (i + 1 == nx) ? 0 : i + 1;
                const double d_ey = eyr[ip] - eyr[i];
                double curl;
                if (p >= 0) {
                    double *ps = psi_c + (int64_t)p * nx + i;
                    *ps = *ps * cb[p];
                    *ps = *ps + cc[p] * d_ex / dx;
                    curl = d_ey / dx + d_ex / (ck[p] * dx) + *ps;
                } else {
                    curl = (d_ey + d_ex) / dx;
                }
                hzr[i] = hzr[i] - ch * curl;
            }
        }
        {
            const double c = ph_h[2 * n], s = ph_h[2 * n + 1];
            const double *hr = hz + (int64_t)a->jr * nx, *ht = hz + (int64_t)a->jt * nx;
            for (int64_t i = 0; i < nx; ++i) {
                dft_hr[2 * i] += hr[i] * c;
                dft_hr[2 * i + 1] += hr[i] * s;
                dft_ht[2 * i] += ht[i] * c;
                dft_ht[2 * i + 1] += ht[i] * s;
            }
        }

        /* E^n -> E^{n+1} */
#pragma omp parallel for schedule(static) num_threads(a->threads)
        for (int64_t j = 0; j < ny; ++j) {
            const double *hzr = hz + j * nx;
            double *exr = ex + j * nx;
            double *eyr = ey + j * nx;
            if (j >= 1) {
                const int32_t p = pml_x_idx[j];
                const double *cxr = cex + j * nx, *cxc = cex_curl + j * nx;
                for (int64_t i = 0; i < nx; ++i) {
                    double d_hz = hzr[i] - hzr[i - nx];
                    if (a->tfsf && j == a->js)
                        d_hz = d_hz - hin;
                    double term;
                    if (p >= 0) {
                        double *ps = psi_x + (int64_t)p * nx + i;
                        *ps = *ps * xb[p];
                        *ps = *ps + xc[p] * d_hz / dx;
                        term = d_hz / (xk[p] * dx) + *ps;
                    } else {
                        term = d_hz / dx;
                    }
                    exr[i] = cxr[i] * exr[i] - cxc[i] * term;
                }
            }
            const double *cyr = cey + j * nx, *cyc = cey_curl + j * nx;
            for (int64_t i = 0; i < nx; ++i) {
                const int64_t im = (i == 0) ? nx - 1 : i - 1;
                const double d_hz_x = hzr[i] - hzr[im];
                eyr[i] = cyr[i] * eyr[i] - cyc[i] * d_hz_x / dx;
            }
        }
        {
            const double c = ph_e[2 * n], s = ph_e[2 * n + 1];
            const double *r0 = ex + (int64_t)a->jr * nx, *t0 = ex + (int64_t)a->jt * nx;
            for (int64_t i = 0; i < nx; ++i) {
                const double er = 0.5 * (r0[i] + r0[nx + i]);
                const double et = 0.5 * (t0[i] + t0[nx + i]);
                dft_er[2 * i] += er * c;
                dft_er[2 * i + 1] += er * s;
                dft_et[2 * i] += et * c;
                dft_et[2 * i + 1] += et * s;
            }
        }
    }
    return 0;
}
