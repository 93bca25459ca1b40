/*
 * libfdtd: 2D FDTD (S: TMz, P: TEz) of segmented leaf cross-sections on one
 * GPU (sm_103a).
 *
 * Problem statement (arXiv 2512.17132, Sec. 2.1 and Sec. 2.6): given a 2D
 * segmented cross-section (a label map), the grid step h and time step dt,
 * the complex index n~ = n + i kappa of every tissue label at the run's
 * wavelength and a normally incident plane wave, return the reflectance R
 * and transmittance T at that wavelength.
 *
 * Discrete system (the same one the FP64 oracle implements):
 *   - TMz Yee leapfrog of Sec. 2.3: Ez at cell centres (times n+1/2), Hx on
 *     the top edge and Hy on the left edge of each cell (times n). Row j = 0
 *     is the top row; rows grow along the incident wave (s = -y). Each step
 *     updates Ez first, then Hx and Hy.
 *   - Per-cell lossy coefficients (Sec. 2.2, Sec. 2.3): eps_r = n^2 - k^2,
 *     sigma = 2 w0 eps0 n k, b = sigma dt/(2 eps0 eps_r),
 *     Ez <- (1-b)/(1+b) Ez + dt/(eps0 eps_r (1+b)) curl H.
 *   - Periodic columns (Sec. 2.4); a CFS-CPML of pml_cells rows at the top
 *     and at the bottom (replacing the paper's split-field PML).
 *   - TF/SF plane-wave source (Sec. 2.5): Ez rows >= tfsf_row and Hx rows
 *     > tfsf_row hold the total field. The incident wave is the echo-free
 *     1D air lattice driven by a hard source s(t) at its cell 0 and read at
 *     its cell/edge 1.
 *   - Running DFTs at w0 of Ez (rows r_row, t_row) and of the row-averaged
 *     Hx (Sec. 2.6) give Poynting fluxes; R and T are normalised by the same
 *     run on an empty (all-air) domain, which the library runs alongside.
 *   - P polarisation (fdtd_source.polarization = FDTD_POL_P) runs the TEz
 *     leapfrog of Sec. 2.3 instead: Hz at cell centres (times n+1/2), Ex on
 *     the top and Ey on the left edge of each cell (times n); each step
 *     updates Hz, then Ex and Ey. The loss coefficients C_e, C_h act on the
 *     E components, so they live on the edges; an edge takes the mean eps_r
 *     and sigma of the two cells it separates. The TF/SF line, CPML, monitors
 *     (DFT of Hz and of the row-averaged Ex) and the empty-domain run follow
 *     the S case with E and H exchanged.
 *
 * Storage on the device is FP32 with H kept as eta0*H; every field exchanged
 * through this interface is in SI units (V/m and A/m), FP32, dense row-major
 * (ny rows of nx values, x fastest), and may be host or device memory. The
 * three field arrays of a handle are (Ez, Hx, Hy) for S polarisation and
 * (Hz, Ex, Ey) for P polarisation: the centre field, the top-edge field and
 * the left-edge field.
 *
 * All functions return FDTD_OK (0) or a negative FDTD_E* code; the message
 * of the last failure on a handle is fdtd_last_error(handle), and failures
 * of fdtd_create (no handle yet) are reported by fdtd_last_error(NULL) on
 * the calling thread. Calls on one handle must not overlap (one host thread
 * at a time); different handles are independent.
 */
#ifndef LIBFDTD_H
#define LIBFDTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDTD_OK 0
#define FDTD_EINVAL (-1)    /* invalid argument (message says which) */
#define FDTD_ENOMEM (-2)    /* device or host allocation failed */
#define FDTD_ECUDA (-3)     /* a CUDA call failed */
#define FDTD_EUNSTABLE (-4) /* the watchdog saw a non-finite field */
#define FDTD_EBOUNDS (-5)   /* debug builds (FDTD_DEBUG_BOUNDS): an in-kernel index check
                               failed (the access was skipped) or a guard band around a
                               device buffer was overwritten; the message names the sites */
#define FDTD_ESTATE (-6)    /* state buffer of the wrong size or layout */

/* Grid and row layout. Rows: 0 <= pml_cells; pml_cells <= r_row < tfsf_row;
 * tfsf_row < t_row; t_row + 1 < ny - pml_cells. The Courant number
 * c0 dt / dx must not exceed 1/sqrt(2) (the 2D CFL limit of Sec. 2.3).
 * CPML grading at depth d (cells, 0 at the interface, pml_cells at the outer
 * wall): sigma = pml_sigma_max (d/L)^m, kappa = 1 + (pml_kappa_max-1)(d/L)^m,
 * alpha = pml_alpha_max (1 - d/L), with m = pml_order. */
typedef struct fdtd_grid {
    int32_t nx, ny;          /* columns (periodic) and rows */
    double dx, dt;           /* cell size [m] and time step [s] */
    int32_t pml_cells;       /* CPML rows at the top and at the bottom */
    int32_t tfsf_row;        /* first total-field Ez row */
    int32_t r_row;           /* reflection monitor row (scattered field) */
    int32_t t_row;           /* transmission monitor row (total field) */
    double pml_order;        /* polynomial grading order m */
    double pml_sigma_max;    /* [S/m] */
    double pml_kappa_max;    /* >= 1 */
    double pml_alpha_max;    /* [S/m] */
} fdtd_grid;

/* Complex refractive index n + i k of one label at the run's wavelength. */
typedef struct fdtd_material {
    double n, k;
} fdtd_material;

/* Incident waveform s(t) at the hard-source cell of the incident lattice:
 * kind 0: exp(-(t-t0)^2/(2 tau^2)) sin(w0 (t-t0)) with amplitude-spectrum
 *         FWHM = rel_bandwidth * f0, tau = 2 sqrt(2 ln 2)/(2 pi rel_bandwidth f0),
 *         t0 = t0_over_tau * tau;
 * kind 1: sin(w0 t) under a raised-cosine ramp over the first 10 periods;
 * kind 2: no incident wave (fields come from fdtd_set_fields/load_state).
 * w0 = 2 pi c0 / lambda0 is also the DFT frequency and the frequency at
 * which sigma is evaluated. */
#define FDTD_POL_S 0  /* TMz: Ez, Hx, Hy */
#define FDTD_POL_P 1  /* TEz: Hz, Ex, Ey (at most 16 labels; labels, not maps) */

typedef struct fdtd_source {
    int32_t kind;
    int32_t polarization;    /* FDTD_POL_S or FDTD_POL_P (Sec. 2.1: the two runs
                                of unpolarised light) */
    double lambda0;          /* [m] */
    double rel_bandwidth;
    double t0_over_tau;
} fdtd_source;

typedef struct fdtd_handle fdtd_handle;

/* Per-handle counters. stencil_ms sums CUDA-event time over the stencil
 * launches when FDTD_OPT_TIMING is on (0 otherwise); it is complete after
 * fdtd_flux or fdtd_synchronize. */
typedef struct fdtd_stats {
    int64_t steps;            /* time steps taken */
    int64_t stencil_launches; /* launches of the main field-update kernel */
    int64_t total_launches;   /* all kernel launches of this handle */
    double stencil_ms;        /* event-timed duration of those launches */
    int32_t kernel;           /* stencil in use: 1 naive, 2 temporally blocked */
    int32_t block_steps;      /* steps per blocked launch */
    int32_t seg_rows;         /* rows per warp task of the blocked kernel */
    int32_t variant;          /* blocked-kernel code shape in use (FDTD_OPT_VARIANT) */
    int32_t graph;            /* batches: 1 when captured CUDA graphs replay the launches */
} fdtd_stats;

/* Options for fdtd_set_option. */
#define FDTD_OPT_KERNEL 1      /* 0 auto, 1 per-half-step kernels, 2 temporally blocked */
#define FDTD_OPT_BLOCK_STEPS 2 /* steps per blocked launch, 1..8 (default 8) */
#define FDTD_OPT_SEG_ROWS 3    /* rows per warp task of the blocked kernel (0 = auto) */
#define FDTD_OPT_TIMING 4      /* 1: time stencil launches with CUDA events */
#define FDTD_OPT_WATCHDOG 5    /* check fields for non-finite values every N steps (0 off) */
#define FDTD_OPT_VARIANT 6     /* blocked-kernel code shape: 0 one row per loop trip with a register
                                  prefetch, 1 two rows per trip, 2 rows streamed through a
                                  shared-memory ring by cp.async, two lean rows per trip, 3 the
                                  ring with one row per trip, built under a 224-register cap,
                                  5 shape 2 with paired FP32 instructions (at most 16 labels;
                                  S adds a label-pair coefficient table). Default: 5 where
                                  allowed, else 2; P handles run shapes 2, 3 and 5; 4 and 6 are
                                  internal (EINVAL) */
#define FDTD_OPT_GRAPH 7       /* batches: replay captured CUDA graphs of launch chunks (default 1) */
#define FDTD_OPT_PLAN_WEIGHT 8 /* segment planner: cost of a general-path iteration of the blocked
                                  kernel in lean iterations, times 1000 (0: the measured defaults,
                                  12 for S and 8.5 for P, and for fdtd_backward 8 for the
                                  recompute and 10 for the reverse kernel); batches take each
                                  handle's value */
#define FDTD_OPT_ADJ_BLOCK 11    /* fdtd_backward: reverse steps per launch of the temporally
                                  blocked reverse kernel, 1..4 (default 3), or 0 for one launch
                                  pair per reverse step; labelled handles with nx % 4 == 0 (the
                                  others always take one step per launch); same gradients bit
                                  for bit */
#define FDTD_OPT_DEBUG_TABLE_LIMIT 9 /* debug builds only (else FDTD_EINVAL): the index checks
                                  admit only this many incident/phase table entries (0: all
                                  allocated), so a longer run trips the table check without
                                  any out-of-range access; tests the checks end to end */
#define FDTD_OPT_DEBUG_POKE_GUARD 10 /* debug builds only (else FDTD_EINVAL): value 1 writes one
                                  byte into the guard band behind the Ez buffer, which the
                                  next synchronising call must report as FDTD_EBOUNDS */

/* Create a simulation. grid, labels (ny*nx uint8, values < n_labels), table
 * (n_labels entries, n > k >= 0) and source are copied; the caller keeps
 * ownership of its buffers. labels may be host or device memory.
 * cuda_stream: a cudaStream_t on the current device, or NULL for a stream
 * owned by the handle. Device memory (about 2 x 12 bytes per cell plus the
 * label map) is allocated here. The Ez rows tfsf_row-1 and tfsf_row must be
 * air (n = 1, k = 0) so that the injected wave matches the air lattice.
 * Errors: FDTD_EINVAL (layout, Courant number, labels, table), FDTD_ENOMEM,
 * FDTD_ECUDA. On success *out is a new handle; on failure *out is NULL. */
int fdtd_create(const fdtd_grid* grid, const uint8_t* labels,
                const fdtd_material* table, int32_t n_labels,
                const fdtd_source* source, void* cuda_stream,
                fdtd_handle** out);

/* As fdtd_create, with per-cell materials instead of labels: eps_r and sigma
 * (ny*nx doubles each, [S/m] for sigma, host or device, copied) at the run's
 * wavelength. Rows tfsf_row-1 and tfsf_row must be air (eps_r = 1,
 * sigma = 0). Such handles step with the per-half-step kernels. */
int fdtd_create_maps(const fdtd_grid* grid, const double* eps_r, const double* sigma,
                     const fdtd_source* source, void* cuda_stream, fdtd_handle** out);

/* Advance by `steps` (>= 0) leapfrog steps (Sec. 2.3), accumulating the
 * monitor DFTs, and the empty-domain reference run by the same steps.
 * Asynchronous on the handle's stream; host work (the incident-wave tables)
 * overlaps the device work. */
int fdtd_run(fdtd_handle* h, int64_t steps);

/* Return to step 0: zero the fields, CPML auxiliaries, DFT accumulators and
 * the empty-domain run; geometry, materials and tables are kept. Async. */
int fdtd_reset(fdtd_handle* h);

/* Wait for all work of the handle; reports watchdog and timeout flags. */
int fdtd_synchronize(fdtd_handle* h);

/* Reflectance and transmittance at lambda0 from the DFTs accumulated so far
 * (Sec. 2.6, Poynting form): R = P_up(r_row)/P_inc, T = P_down(t_row)/P_inc,
 * P_inc = nx * P_down(t_row) of the empty-domain run. Synchronises. Before
 * the incident pulse has reached t_row, P_inc is 0 and R, T are not finite
 * (IEEE division); fdtd_flux_raw gives the powers themselves. */
int fdtd_flux(fdtd_handle* h, double* R, double* T);

/* The three fluxes behind R and T in W/m (per unit z length):
 * out[0] = P_up at r_row, out[1] = P_down at t_row, out[2] = P_inc. */
int fdtd_flux_raw(fdtd_handle* h, double out[3]);

/* Running DFT accumulators (Sec. 2.6) in SI units: 4 rows of nx complex
 * values, each stored as (re, im) doubles (8*nx doubles in total, host or
 * device), in the order Ez(r_row), Hx(r_row), Ez(t_row), Hx(t_row); the Hx
 * rows average the edges row and row+1. P polarisation: Hz(r_row),
 * Ex(r_row), Hz(t_row), Ex(t_row), with the Ex rows averaged alike. */
int fdtd_get_dft(fdtd_handle* h, double* out);

/* CW steady state (Sec. 2.6: the fields are sampled over whole periods once
 * they are periodic): zero the running DFTs of the handle and of its
 * empty-domain run, so that the next fdtd_run steps form the window. With a
 * ramped CW source (kind 1), run past the ramp and the transient, call this,
 * then run an integer number of periods (lambda0 / (c0 dt) steps each).
 * Synchronous. */
int fdtd_reset_dft(fdtd_handle* h);

/* Bloch-order decomposition of the monitor lines (Sec. 2.6). The fields are
 * periodic in x with period L = nx dx, so each DFT line expands as
 * sum_m X_m exp(i 2 pi m x / L). For m = -m_max..m_max (2 m_max + 1 <= nx),
 * out[8 (m + m_max) + q] (host memory, 8 (2 m_max + 1) doubles) holds:
 *   q = 0, 1: order m's share of the Poynting fluxes, P_up,m / P_inc and
 *             P_down,m / P_inc (Parseval: the shares of all nx orders sum to
 *             R and T of fdtd_flux; evanescent orders carry none);
 *   q = 2, 3: the paper's |E_ref,m|^2 / |E_inc,0|^2 and |E_trs,m|^2 /
 *             |E_inc,0|^2 with E = Ez (S) or the row-averaged Ex (P) and
 *             E_inc,0 from the empty-domain run;
 *   q = 4, 5: the same times the obliquity factor w_m (the power an oblique
 *             order carries per |E_m|^2 relative to order 0, which the
 *             paper's sum leaves out);
 *   q = 6:    w_m = sin(k_y,m dx)/sin(k_y,0 dx) for S, its inverse for P,
 *             0 for evanescent orders;
 *   q = 7:    k_y,m dx from the 2D lattice dispersion relation
 *             sin^2(k_y dx/2) = sin^2(w0 dt/2)/S^2 - sin^2(pi m/nx), NaN when
 *             the order is evanescent.
 * The order amplitudes are computed on the device in FP64. Synchronous.
 * fdtd_bloch_propagating returns the largest M such that every |m| <= M is
 * a propagating order (and 2M + 1 <= nx), or FDTD_EINVAL for NULL. */
int fdtd_bloch_orders(fdtd_handle* h, int32_t m_max, double* out);
int32_t fdtd_bloch_propagating(const fdtd_handle* h);

/* Read or overwrite the fields (SI, FP32, ny*nx each, host or device; a NULL
 * pointer skips that field): (Ez, Hx, Hy) for S polarisation, (Hz, Ex, Ey)
 * for P polarisation. Row 0 of the top-edge field (Hx, or Ex) is the fixed
 * top wall and reads 0; fdtd_set_fields forces it to 0. Synchronous. */
int fdtd_get_fields(fdtd_handle* h, float* ez, float* hx, float* hy);
int fdtd_set_fields(fdtd_handle* h, const float* ez, const float* hx,
                    const float* hy);

/* Complete simulation state (fields, CPML auxiliaries, DFT accumulators,
 * empty-domain run, step count) for checkpoint / restart. The buffer (host
 * or device) must hold fdtd_state_bytes(h) bytes; load requires a handle
 * created with the same grid. */
size_t fdtd_state_bytes(const fdtd_handle* h);
int fdtd_save_state(fdtd_handle* h, void* buf, size_t bytes);
int fdtd_load_state(fdtd_handle* h, const void* buf, size_t bytes);

/* Tuning and instrumentation switches (FDTD_OPT_*). */
int fdtd_set_option(fdtd_handle* h, int32_t option, int64_t value);
int fdtd_get_stats(fdtd_handle* h, fdtd_stats* out);

/* Message of the last failure on h (or of fdtd_create on this thread when h
 * is NULL); "" if none. Valid until the next call on h. */
const char* fdtd_last_error(const fdtd_handle* h);

/* Release the handle and its device memory (waits for its work). NULL is a
 * no-op. */
void fdtd_destroy(fdtd_handle* h);

/* Discrete adjoint (reverse-mode gradient of the leapfrog recursion) of
 * J = wR R + wT T (R, T as in fdtd_flux).
 * fdtd_forward_checkpointed: reset, run `steps` steps and keep the full state
 * every `every` steps on the device (about 12 bytes per cell each).
 * fdtd_backward: for J at the end of that run, dJ/d(eps_r) and dJ/d(sigma)
 * per cell (ny*nx doubles each, host or device, NULL to skip) and, for
 * labelled handles, dJ/dn and dJ/dk per label (n_labels pairs, host or
 * device, NULL to skip); out = {J, R, T} (may be NULL). Segment by segment
 * (last first) the steps are recomputed from their checkpoint, storing for
 * each step the two forward factors of the gradient sums (Ez before the
 * update and the factor of cb in it) on a device tape (about 8*every bytes
 * per cell plus two states; the handle keeps it for the next fdtd_backward
 * of the same size and fdtd_destroy frees it), and the transpose of every
 * update is applied in reverse order; per-segment FP32 sums are accumulated
 * in FP64. The handle keeps its final forward
 * state. FDTD_ESTATE if no checkpointed run precedes or no incident power
 * reached t_row; FDTD_EINVAL for P-polarised handles (the adjoint covers
 * the S case). Synchronises. */
int fdtd_forward_checkpointed(fdtd_handle* h, int64_t steps, int32_t every);
int fdtd_backward(fdtd_handle* h, double wR, double wT, double* g_eps, double* g_sigma,
                  double* g_label, double out[3]);

/* Pick the blocked kernel's steps per launch, code shape and segment height
 * for this handle's grid by timing `trial_launches` launches of each
 * candidate on the current state. The trial launches write only scratch
 * (the other ping-pong buffers and a dummy monitor sink), so the simulation
 * state is unchanged. The choice is remembered per (nx, ny, pml_cells,
 * device) for later handles. Synchronises. */
int fdtd_autotune(fdtd_handle* h, int32_t trial_launches);

/* Row segments of the blocked kernel's load-balancing plan (host only; no
 * device is touched, so it also runs where no GPU is present). The paper
 * has no counterpart: this is the planner of this implementation's warp
 * tasks, exposed for inspection and tests. For grid g (its rows checked as
 * by fdtd_create), about ny / seg_rows segments (seg_rows below
 * block_steps + 1 is raised to it), block_steps K in 1..8 and polarisation
 * FDTD_POL_S or FDTD_POL_P it writes the row boundaries
 * 0 = b[0] < b[1] < ... < b[n] = ny to out[0..n] and returns n + 1.
 * The cuts minimise, to within a quarter of a lean iteration, the largest
 * estimated segment cost over plans of at most N = round(ny / seg_rows)
 * segments; segments are then split at their cost midpoints, costliest
 * first, while fewer than N exist and one can be split. Iteration t of the
 * warp task of segment [y0, y1) (t from y0 - K, or from 0 for the first
 * segment, to y1 + K - 1) costs 1 when the rows t-K..t-1 it updates are
 * all in 1..ny-P-1, outside the top CPML rows 0..P-1, and miss tfsf_row,
 * r_row, r_row + 1, t_row and t_row + 1; otherwise it costs a fixed
 * per-polarisation weight (the general path). Every inner boundary is >= K
 * and differs from r_row + 1 and t_row + 1. Errors: FDTD_EINVAL for a bad
 * grid, K or polarisation, or cap < n + 1; FDTD_ENOMEM when host memory
 * runs out (message in fdtd_last_error(NULL)). The handle path cuts the
 * same plan for the segment height its wave model picks
 * (fdtd_stats.seg_rows). */
int fdtd_plan_segments(const fdtd_grid* g, int32_t seg_rows, int32_t block_steps,
                       int32_t polarization, int32_t* out, int32_t cap);

/* Batched runs of independent simulations (the paper runs one simulation
 * per wavelength, polarisation and slice, Sec. 2.2 and Sec. 4; here they
 * share the GPU). A batch groups existing handles (same device, nx % 4 == 0
 * each; the handles must outlive the batch). fdtd_batch_run advances every
 * handle by `steps` in lockstep (all handles of one batch share one
 * polarisation, else FDTD_EINVAL): one blocked-kernel launch per K steps
 * covers the warp tasks of all simulations, the empty-domain runs go as one
 * launch on a side stream, and full chunks of launches are captured once
 * into a CUDA graph and replayed (FDTD_OPT_GRAPH). The results are exactly
 * those of running each handle alone; read them with fdtd_flux etc. on each
 * handle. Work is ordered after earlier work on every handle's streams and
 * later work on them waits for the batch. Options: FDTD_OPT_BLOCK_STEPS,
 * FDTD_OPT_SEG_ROWS, FDTD_OPT_VARIANT, FDTD_OPT_TIMING, FDTD_OPT_GRAPH.
 * fdtd_batch_autotune times candidate launch shapes on the whole batch like
 * fdtd_autotune (state unchanged). Stats: graph = 1 when a graph is in use.
 * Errors of fdtd_batch_create are reported by fdtd_batch_last_error(NULL). */
typedef struct fdtd_batch fdtd_batch;
int fdtd_batch_create(fdtd_handle* const* hs, int32_t n, fdtd_batch** out);
int fdtd_batch_set_option(fdtd_batch* b, int32_t option, int64_t value);
int fdtd_batch_autotune(fdtd_batch* b, int32_t trial_launches);
int fdtd_batch_run(fdtd_batch* b, int64_t steps);
int fdtd_batch_get_stats(fdtd_batch* b, fdtd_stats* out);
const char* fdtd_batch_last_error(const fdtd_batch* b);
void fdtd_batch_destroy(fdtd_batch* b);

/* Allocation-free stepping. The paper has no counterpart: this is an
 * interface for callers that may not call cudaMalloc where they step the
 * fields, such as a plug-in confined to a device-memory budget that its host
 * framework hands out, or a process whose device memory belongs to another
 * runtime's allocator (a framework's caching allocator that already holds
 * the GPU). fdtd_create and fdtd_run allocate their state and tables; this
 * call uses only buffers the caller owns plus a static scratch array.
 *
 * Advances a source-free field state by `steps` (1..8) leapfrog steps with
 * the temporally blocked kernel (code shape 5 for at most 16 labels, else
 * 2) on `cuda_stream` (NULL = legacy stream), and allocates nothing: the
 * kernel's scratch (segment table, coefficient and CPML tables, zeroed
 * source tables, a sink for monitor sums) lives in one static 8 MiB device
 * array per GPU, held by every GPU that loads the library until the process
 * exits. Grids needing more scratch (roughly nx > 130000, or pml_cells > 64)
 * are rejected with FDTD_EINVAL and a message.
 *   grid: layout as for fdtd_create (nx % 4 == 0 required); table/n_labels/
 *     lambda0: materials at the wavelength (coefficients as in fdtd_create);
 *   labels: device, ny*nx uint8, values < n_labels (not checked here),
 *     4-byte aligned;
 *   in[5], out[5]: device buffers {Ez, eta0*Hx, eta0*Hy, psi_E, psi_H},
 *     16-byte aligned: fields dense ny*nx FP32 (Ez in V/m, H scaled by
 *     eta0 = mu0 c0, i.e. also V/m), CPML carries dense (2*pml_cells)*nx
 *     FP32 (top rows first, zero at the start of a run); outputs must not
 *     alias inputs; the caller owns all of them. Hx row 0 stays as given
 *     (the fixed top edge).
 *   err/err_len: optional buffer for a message on failure.
 * A call launches two kernels on the stream: the first copies the tables,
 * computed on the host and passed by value as its launch parameters, into
 * the scratch array and clears its zeroed parts; the second steps the
 * fields. No host memory is read after the call returns, and the call does
 * not wait for earlier work on the stream.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture begins.
 * Every call shares the one array and overwrites it, so calls that overlap
 * on the GPU race; nothing in it needs to persist between calls.
 * Returns FDTD_OK, FDTD_EINVAL or FDTD_ECUDA; asynchronous on success. */
int fdtd_blocked_advance_noalloc(const fdtd_grid* grid, const uint8_t* labels,
                                 const fdtd_material* table, int32_t n_labels,
                                 double lambda0, const float* const* in,
                                 float* const* out, int32_t steps,
                                 void* cuda_stream, char* err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* LIBFDTD_H */
