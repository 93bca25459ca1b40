"""Plain FP64 reference of the 2D TMz Yee FDTD loop (S-polarisation).

TEST INFRASTRUCTURE: a slow, direct restatement of the discrete method, used
only to check the CUDA library. Everything is SI and float64; one array
statement per update equation, no blocking, fusion or reordering.

Discrete system (Sec. 2.3 TMz equations, rows counted downward):
  * x is the periodic horizontal axis (column i), s = -y the vertical axis
    pointing along the incident wave (row j = 0 at the top).
  * Ez[j, i] sits at the cell centre ((i+1/2) dx, (j+1/2) dx) at times n+1/2;
    Hx[j, i] on the top edge (i+1/2, j) and Hy[j, i] on the left edge
    (i, j+1/2), both at integer times n. Hx[0] and the virtual Hx[ny] stay 0.
  * Because y = -s, the paper's -dHx/dy becomes +dHx/ds, so the Ez update
    reads the edge pair (Hx[j+1] - Hx[j]) that brackets cell j; the paper's
    printed pair (Hx_j - Hx_{j-1}) is off by one row and is read this way.
  * C_h in Sec. 2.3 omits the factor dt / (eps0 eps_r); it is restored here:
    Ez <- C_e Ez + C_h dt/(eps0 eps_r) * curl H, with C_e = (1-b)/(1+b),
    C_h = 1/(1+b), b = sigma dt / (2 eps0 eps_r).
  * Lateral boundaries are periodic (Sec. 2.4): i-1 and i+1 wrap modulo nx.
  * Top and bottom carry a CFS-CPML (Roden-Gedney convolutional PML) of
    pml_cells rows in place of the paper's split-field PML (Sec. 2.4).
  * A normally incident plane wave enters through a TF/SF line (Sec. 2.5):
    Ez rows >= tfsf_row and Hx rows > tfsf_row are total field.
  * Running DFTs at rows r_row (scattered field, above the source) and t_row
    (total field, below the leaf) give Poynting fluxes (Sec. 2.6), and
    R, T are normalised by the same run on an empty (all-air) domain.

Parity pins for every function live in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import math

import numpy as np

C0 = 299_792_458.0
MU0 = 4.0e-7 * math.pi
EPS0 = 1.0 / (MU0 * C0 * C0)
ETA0 = MU0 * C0

SOURCE_PULSE, SOURCE_CW, SOURCE_NONE = 0, 1, 2


def eps_sigma(n, k, omega):
    """Complex index -> (eps_r, sigma) at angular frequency omega (Sec. 2.2):
    eps_r = n^2 - kappa^2, sigma = omega eps0 Im(n~^2) = 2 omega eps0 n kappa."""
    n = np.asarray(n, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    return n * n - k * k, 2.0 * omega * EPS0 * n * k


def lossy_coefficients(eps_r, sigma, dt):
    """Time-averaged loss coefficients of Sec. 2.3:
    C_e = (1 - b)/(1 + b), C_h = 1/(1 + b), b = sigma dt / (2 eps0 eps_r)."""
    b = sigma * dt / (2.0 * EPS0 * eps_r)
    return (1.0 - b) / (1.0 + b), 1.0 / (1.0 + b)


def cpml_profile(depth, thickness, order, sigma_max, kappa_max, alpha_max, dt):
    """CFS-CPML recursion coefficients at a depth (cells) into a layer.

    depth is measured from the interior interface (0) to the outer wall
    (thickness). Polynomial grading sigma = sigma_max (d/L)^m,
    kappa = 1 + (kappa_max - 1)(d/L)^m, and alpha = alpha_max (1 - d/L);
    b = exp(-(sigma/kappa + alpha) dt/eps0),
    c = sigma (b - 1) / (sigma kappa + kappa^2 alpha)  (0 where sigma = 0).
    Returns (b, c, kappa) arrays.
    """
    x = np.asarray(depth, dtype=np.float64) / float(thickness)
    sig = sigma_max * x ** order
    kap = 1.0 + (kappa_max - 1.0) * x ** order
    alp = alpha_max * (1.0 - x)
    b = np.exp(-(sig / kap + alp) * dt / EPS0)
    den = sig * kap + kap * kap * alp
    c = np.where(sig > 0.0, sig * (b - 1.0) / np.where(den > 0.0, den, 1.0), 0.0)
    return b, c, kap


def source_waveform(kind, t, lambda0, rel_bandwidth=0.1, t0_over_tau=5.0):
    """Incident waveform s(t) in V/m.

    kind 0: Gaussian-modulated sinusoid exp(-(t-t0)^2/(2 tau^2)) sin(w0 (t-t0)),
            with the amplitude-spectrum FWHM equal to rel_bandwidth * f0:
            sigma_f = rel_bandwidth f0 / (2 sqrt(2 ln 2)), tau = 1/(2 pi sigma_f),
            t0 = t0_over_tau * tau.
    kind 1: sin(w0 t) under a raised-cosine ramp over the first 10 periods.
    kind 2: no source (s = 0).
    """
    f0 = C0 / lambda0
    w0 = 2.0 * math.pi * f0
    if kind == SOURCE_PULSE:
        sigma_f = rel_bandwidth * f0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))
        tau = 1.0 / (2.0 * math.pi * sigma_f)
        t0 = t0_over_tau * tau
        return math.exp(-((t - t0) ** 2) / (2.0 * tau * tau)) * math.sin(w0 * (t - t0))
    if kind == SOURCE_CW:
        t_ramp = 10.0 / f0
        ramp = 1.0 if t >= t_ramp else 0.5 * (1.0 - math.cos(math.pi * t / t_ramp))
        return ramp * math.sin(w0 * t)
    return 0.0


class IncidentLine:
    """The incident plane wave of the TF/SF source (Sec. 2.5) on a 1D lattice.

    A semi-infinite air lattice with the same dx and dt as the 2D grid: cell
    k holds Ez at (k+1/2) dx, edge k holds Hx at k dx. Cell 0 is a hard
    source, Ez[0]^{n+1/2} = s((n+1/2) dt). The incident fields handed to the
    TF/SF line are Ez at cell 1 (time n+1/2) and Hx at edge 1 (time n).
    Signals move at most one cell per step on this lattice, so keeping it
    longer than the number of steps taken makes it exactly echo-free.
    """

    def __init__(self, dx, dt, kind, lambda0, rel_bandwidth, t0_over_tau):
        self.dx, self.dt = dx, dt
        self.kind, self.lambda0 = kind, lambda0
        self.bw, self.t0 = rel_bandwidth, t0_over_tau
        self.ez = np.zeros(64)
        self.hx = np.zeros(64)
        self.n = 0

    def h_inc(self):
        """Hx at edge 1, time n."""
        return self.hx[1]

    def advance_e(self):
        """Ez: n-1/2 -> n+1/2 (air: C_e = 1, C_h = 1)."""
        if self.n + 8 >= len(self.ez):
            self.ez = np.concatenate([self.ez, np.zeros(len(self.ez))])
            self.hx = np.concatenate([self.hx, np.zeros(len(self.hx))])
        hx_next = np.append(self.hx[1:], 0.0)            # Hx[k+1]
        self.ez[1:] += self.dt / (EPS0 * self.dx) * (hx_next[1:] - self.hx[1:])
        self.ez[0] = source_waveform(self.kind, (self.n + 0.5) * self.dt,
                                     self.lambda0, self.bw, self.t0)

    def e_inc(self):
        """Ez at cell 1, time n+1/2."""
        return self.ez[1]

    def advance_h(self):
        """Hx: n -> n+1."""
        self.hx[1:] += self.dt / (MU0 * self.dx) * (self.ez[1:] - self.ez[:-1])
        self.n += 1


class TMzOracle:
    """FP64 TMz FDTD on one grid (fields in SI units).

    spec: any object with the attributes nx, ny, dx, dt, pml_cells, pml_order,
    pml_sigma_max, pml_kappa_max, pml_alpha_max, tfsf_row, r_row, t_row,
    lambda0, source_kind, rel_bandwidth, t0_over_tau, labels (ny, nx) and
    materials (n_labels, 2) = (n, kappa). eps_r / sigma maps (ny, nx) may be
    given instead of labels + materials.
    """

    def __init__(self, spec, eps_r=None, sigma=None):
        self.nx, self.ny = int(spec.nx), int(spec.ny)
        self.dx, self.dt = float(spec.dx), float(spec.dt)
        self.P = int(spec.pml_cells)
        self.js, self.jr, self.jt = int(spec.tfsf_row), int(spec.r_row), int(spec.t_row)
        self.omega = 2.0 * math.pi * C0 / spec.lambda0
        courant = C0 * self.dt / self.dx
        if courant > 1.0 / math.sqrt(2.0) * (1.0 + 1e-12):
            raise ValueError(f"Courant number {courant} exceeds the 2D CFL limit 1/sqrt(2) (Sec. 2.3)")
        if eps_r is None:
            mats = np.asarray(spec.materials, dtype=np.float64)
            lab = np.asarray(spec.labels)
            eps_r, sigma = eps_sigma(mats[lab, 0], mats[lab, 1], self.omega)
        self.eps_r = np.asarray(eps_r, dtype=np.float64).reshape(self.ny, self.nx)
        self.sigma = np.asarray(sigma, dtype=np.float64).reshape(self.ny, self.nx)
        self.ce, ch = lossy_coefficients(self.eps_r, self.sigma, self.dt)
        self.ce_curl = ch * self.dt / (EPS0 * self.eps_r)   # multiplies curl H
        self.ch_curl = self.dt / MU0                         # multiplies curl E
        self.ez = np.zeros((self.ny, self.nx))
        self.hx = np.zeros((self.ny, self.nx))
        self.hy = np.zeros((self.ny, self.nx))
        self._setup_cpml(spec)
        self.inc = IncidentLine(self.dx, self.dt, int(spec.source_kind), spec.lambda0,
                                spec.rel_bandwidth, spec.t0_over_tau)
        self.n = 0
        self.dft = {k: np.zeros(self.nx, dtype=np.complex128)
                    for k in ("e_r", "h_r", "e_t", "h_t")}
        self.tape = None          # list: (Ez^{n-1/2}, curl^n) per step when recording

    # -- CPML ---------------------------------------------------------------
    def _setup_cpml(self, spec):
        P, ny = self.P, self.ny
        prof = lambda d: cpml_profile(d, P, spec.pml_order, spec.pml_sigma_max,
                                      spec.pml_kappa_max, spec.pml_alpha_max, self.dt)
        self.pml_e = []   # (rows, b, c, kappa, psi) for Ez rows in the layers
        self.pml_h = []   # same for Hx rows
        if P <= 0:
            return
        top_e = np.arange(0, P)
        bot_e = np.arange(ny - P, ny)
        top_h = np.arange(1, P)                 # edge P is the interface (depth 0)
        bot_h = np.arange(ny - P + 1, ny)
        for rows, depth in ((top_e, P - top_e - 0.5), (bot_e, bot_e + 0.5 - (ny - P))):
            b, c, k = prof(depth)
            self.pml_e.append((rows, b[:, None], c[:, None], k[:, None],
                               np.zeros((len(rows), self.nx))))
        for rows, depth in ((top_h, (P - top_h).astype(float)),
                            (bot_h, (bot_h - (ny - P)).astype(float))):
            b, c, k = prof(depth)
            self.pml_h.append((rows, b[:, None], c[:, None], k[:, None],
                               np.zeros((len(rows), self.nx))))

    # -- one leapfrog step ---------------------------------------------------
    def step(self):
        dx, js = self.dx, self.js
        h_inc = self.inc.h_inc()                       # H_inc(edge js, n)
        self.inc.advance_e()
        e_inc = self.inc.e_inc()                       # E_inc(cell js, n+1/2)

        # Ez^{n-1/2} -> Ez^{n+1/2}  (Sec. 2.3, TMz Ez equation)
        hx_below = np.zeros_like(self.hx)
        hx_below[:-1] = self.hx[1:]                    # Hx[j+1]; Hx[ny] = 0
        d_hx = hx_below - self.hx                      # Hx[j+1] - Hx[j]
        if self.inc.kind != SOURCE_NONE:
            d_hx[js] -= h_inc                          # TF cell js sees total Hx[js]
        d_hy = np.roll(self.hy, -1, axis=1) - self.hy  # Hy[i+1] - Hy[i] (periodic)
        curl = (d_hy + d_hx) / dx
        for rows, b, c, k, psi in self.pml_e:
            psi *= b
            psi += c * d_hx[rows] / dx
            curl[rows] = d_hy[rows] / dx + d_hx[rows] / (k * dx) + psi
        if self.tape is not None:
            self.tape.append((self.ez, curl))
        self.ez = self.ce * self.ez + self.ce_curl * curl

        tE = (self.n + 0.5) * self.dt
        self.dft["e_r"] += self.ez[self.jr] * np.exp(1j * self.omega * tE)
        self.dft["e_t"] += self.ez[self.jt] * np.exp(1j * self.omega * tE)

        # H^n -> H^{n+1}  (Sec. 2.3, TMz Hx and Hy equations)
        d_ez = self.ez[1:] - self.ez[:-1]              # Ez[j] - Ez[j-1], rows 1..ny-1
        if self.inc.kind != SOURCE_NONE:
            d_ez[js - 1] -= e_inc                      # SF edge js sees scattered Ez[js]
        term = d_ez / dx
        for rows, b, c, k, psi in self.pml_h:
            psi *= b
            psi += c * d_ez[rows - 1] / dx
            term[rows - 1] = d_ez[rows - 1] / (k * dx) + psi
        self.hx[1:] += self.ch_curl * term
        d_ez_x = self.ez - np.roll(self.ez, 1, axis=1)  # Ez[i] - Ez[i-1] (periodic)
        self.hy += self.ch_curl * d_ez_x / dx
        self.inc.advance_h()

        tH = (self.n + 1.0) * self.dt
        ph = np.exp(1j * self.omega * tH)
        self.dft["h_r"] += 0.5 * (self.hx[self.jr] + self.hx[self.jr + 1]) * ph
        self.dft["h_t"] += 0.5 * (self.hx[self.jt] + self.hx[self.jt + 1]) * ph
        self.n += 1

    def run(self, steps):
        for _ in range(int(steps)):
            self.step()
        return self

    def reset_dft(self):
        """Restart the running DFTs at the current step (a CW steady-state
        window, Sec. 2.6: sampling starts once the fields are periodic)."""
        for v in self.dft.values():
            v[:] = 0.0

    # -- state access --------------------------------------------------------
    def fields(self):
        return self.ez.copy(), self.hx.copy(), self.hy.copy()

    def set_fields(self, ez, hx, hy):
        self.ez = np.array(ez, dtype=np.float64).reshape(self.ny, self.nx)
        self.hx = np.array(hx, dtype=np.float64).reshape(self.ny, self.nx)
        self.hy = np.array(hy, dtype=np.float64).reshape(self.ny, self.nx)
        self.hx[0] = 0.0

    def fluxes(self):
        """Time-averaged Poynting fluxes (W/m per unit z-length) at the
        monitor rows: upward at r_row, downward at t_row. The downward
        component of E x H for TMz is -Ez Hx, so
        P_down = -1/2 Re sum_i Ez~ conj(Hx~) dx and P_up = -P_down."""
        d = self.dft
        p_r = 0.5 * np.real(np.sum(d["e_r"] * np.conj(d["h_r"]))) * self.dx
        p_t = 0.5 * np.real(np.sum(d["e_t"] * np.conj(d["h_t"]))) * self.dx
        return p_r, -p_t


def empty_twin(spec):
    """The empty-domain reference run: one column of air with the same rows,
    CPML, source and monitors (an x-uniform field needs a single column)."""
    class _S:
        pass
    s = _S()
    for a in ("ny", "dx", "dt", "pml_cells", "pml_order", "pml_sigma_max",
              "pml_kappa_max", "pml_alpha_max", "tfsf_row", "r_row", "t_row",
              "lambda0", "source_kind", "rel_bandwidth", "t0_over_tau"):
        setattr(s, a, getattr(spec, a))
    s.nx = 1
    s.labels = np.zeros((spec.ny, 1), dtype=np.uint8)
    s.materials = np.array([[1.0, 0.0]])
    return TMzOracle(s)


def run_rt(spec, steps=None):
    """R, T and A = 1 - R - T at lambda0 (Sec. 2.6), with the incident power
    taken from the empty-domain run at t_row and scaled to the nx columns."""
    steps = spec.steps if steps is None else steps
    leaf = TMzOracle(spec).run(steps)
    twin = empty_twin(spec).run(steps)
    p_up, p_down = leaf.fluxes()
    _, p0 = twin.fluxes()
    p_inc = p0 * spec.nx
    R, T = p_up / p_inc, p_down / p_inc
    return dict(R=R, T=T, A=1.0 - R - T, p_up=p_up, p_down=p_down, p_inc=p_inc,
                leaf=leaf, twin=twin)
