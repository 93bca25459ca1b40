"""Plain FP64 reference of the 2D TEz Yee FDTD loop (P-polarisation).

TEST INFRASTRUCTURE: a slow, direct restatement of the discrete method, used
only to check the CUDA library. Everything is SI and float64; one array
statement per update equation, no blocking, fusion or reordering.

Discrete system (Sec. 2.3 TEz equations, rows counted downward, s = -y):
  * Hz[j, i] sits at the cell centre ((i+1/2) dx, (j+1/2) dx) at times n+1/2;
    Ex[j, i] on the top edge (i+1/2, j) and Ey[j, i] on the left edge
    (i, j+1/2), both at integer times n. Ex[0] and the virtual Ex[ny] stay 0
    (electric walls behind the CPML).
  * With d/dy = -d/ds the curl equations read
      dHz/dt = -(1/mu0) (dEy/dx + dEx/ds),
      dEx/dt = -(1/(eps0 eps_r)) dHz/ds - sigma/(eps0 eps_r) Ex,
      dEy/dt = -(1/(eps0 eps_r)) dHz/dx - sigma/(eps0 eps_r) Ey,
    so the Hz update reads the edge pairs (Ey[i+1] - Ey[i]) and
    (Ex[j+1] - Ex[j]) that bracket cell (j, i), and the E updates the centre
    pairs (Hz[j] - Hz[j-1]) and (Hz[i] - Hz[i-1]) that bracket each edge.
  * The loss coefficients C_e, C_h of Sec. 2.3 multiply the E components,
    which live on edges. The paper evaluates them at the edge but does not
    say which material an edge between two cells has; here eps_r and sigma of
    an edge are the arithmetic means of the two cells it separates (the
    complex permittivity averaged along the tangential E component). C_h is
    completed with its missing dt / (eps0 eps_r) factor as in the TMz oracle.
  * Lateral boundaries are periodic (Sec. 2.4), top and bottom carry the same
    CFS-CPML as the TMz oracle: the Hz rows use the cell-centre profile, the
    Ex rows the edge profile.
  * TF/SF line (Sec. 2.5): Hz rows >= tfsf_row and Ex rows > tfsf_row are
    total field. The incident pair comes from a 1D air lattice whose cell 0
    is a hard source eta0 Hz = s((n+1/2) dt), so the incident Ex equals s.
  * Running DFTs of Hz (time n+1/2) and of Ex averaged over the two edges of
    the monitor row (time n+1) give the Poynting fluxes (Sec. 2.6). The
    downward component of E x H for TEz is +Ex Hz.

Parity pins live in tests/test_oracle_tez_pins.py: the exact lattice
solution of x-uniform stacks, the TEz/TMz duality of an all-air domain,
energy conservation and mirror symmetry of a lossless 2D structure.
"""
from __future__ import annotations

import math

import numpy as np

from .fdtd_tmz import (C0, EPS0, ETA0, MU0, SOURCE_NONE, cpml_profile, eps_sigma,
                       lossy_coefficients, source_waveform)


def edge_materials(eps_r, sigma):
    """Material of the Ex (top) and Ey (left) edges: the arithmetic mean of
    the two cells each edge separates. Row 0 of the Ex arrays (the top wall)
    is unused; the Ey edge of column 0 separates columns nx-1 and 0."""
    ex_eps = np.empty_like(eps_r)
    ex_sig = np.empty_like(sigma)
    ex_eps[1:] = 0.5 * (eps_r[:-1] + eps_r[1:])
    ex_sig[1:] = 0.5 * (sigma[:-1] + sigma[1:])
    ex_eps[0] = eps_r[0]
    ex_sig[0] = sigma[0]
    ey_eps = 0.5 * (np.roll(eps_r, 1, axis=1) + eps_r)
    ey_sig = 0.5 * (np.roll(sigma, 1, axis=1) + sigma)
    return ex_eps, ex_sig, ey_eps, ey_sig


class IncidentLineTEz:
    """Incident P-polarised plane wave (Sec. 2.5) on a semi-infinite 1D air
    lattice: cell k holds Hz at (k+1/2) dx, edge k holds Ex at k dx. Cell 0
    is a hard source, eta0 Hz[0]^{n+1/2} = s((n+1/2) dt). The TF/SF line
    receives Hz at cell 1 (time n+1/2) and Ex at edge 1 (time n). The
    lattice grows ahead of the wavefront, so it never echoes."""

    def __init__(self, dx, dt, kind, lambda0, rel_bandwidth, t0_over_tau):
        self.dx, self.dt = dx, dt
        self.kind, self.lambda0 = kind, lambda0
        self.bw, self.t0 = rel_bandwidth, t0_over_tau
        self.hz = np.zeros(64)
        self.ex = np.zeros(64)
        self.n = 0

    def e_inc(self):
        """Ex at edge 1, time n."""
        return self.ex[1]

    def advance_h(self):
        """Hz: n-1/2 -> n+1/2; dHz/dt = -(1/mu0) dEx/ds in air."""
        if self.n + 8 >= len(self.hz):
            self.hz = np.concatenate([self.hz, np.zeros(len(self.hz))])
            self.ex = np.concatenate([self.ex, np.zeros(len(self.ex))])
        ex_next = np.append(self.ex[1:], 0.0)              # Ex[k+1]
        self.hz[1:] -= self.dt / (MU0 * self.dx) * (ex_next[1:] - self.ex[1:])
        self.hz[0] = source_waveform(self.kind, (self.n + 0.5) * self.dt,
                                     self.lambda0, self.bw, self.t0) / ETA0

    def h_inc(self):
        """Hz at cell 1, time n+1/2."""
        return self.hz[1]

    def advance_e(self):
        """Ex: n -> n+1; dEx/dt = -(1/eps0) dHz/ds in air."""
        self.ex[1:] -= self.dt / (EPS0 * self.dx) * (self.hz[1:] - self.hz[:-1])
        self.n += 1


class TEzOracle:
    """FP64 TEz FDTD on one grid (fields in SI units); same spec interface
    as the TMz oracle (labels + (n, kappa) table, or eps_r / sigma maps)."""

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
        ex_eps, ex_sig, ey_eps, ey_sig = edge_materials(self.eps_r, self.sigma)
        self.cex, chx = lossy_coefficients(ex_eps, ex_sig, self.dt)
        self.cey, chy = lossy_coefficients(ey_eps, ey_sig, self.dt)
        self.cex_curl = chx * self.dt / (EPS0 * ex_eps)     # multiplies dHz/ds
        self.cey_curl = chy * self.dt / (EPS0 * ey_eps)     # multiplies dHz/dx
        self.ch_curl = self.dt / MU0                         # multiplies curl E
        self.hz = np.zeros((self.ny, self.nx))
        self.ex = np.zeros((self.ny, self.nx))
        self.ey = np.zeros((self.ny, self.nx))
        self._setup_cpml(spec)
        self.inc = IncidentLineTEz(self.dx, self.dt, int(spec.source_kind), spec.lambda0,
                                   spec.rel_bandwidth, spec.t0_over_tau)
        self.n = 0
        self.dft = {k: np.zeros(self.nx, dtype=np.complex128)
                    for k in ("h_r", "e_r", "h_t", "e_t")}

    def _setup_cpml(self, spec):
        P, ny = self.P, self.ny
        prof = lambda d: cpml_profile(d, P, spec.pml_order, spec.pml_sigma_max,
                                      spec.pml_kappa_max, spec.pml_alpha_max, self.dt)
        self.pml_c = []   # (rows, b, c, kappa, psi) for Hz rows (cell centres)
        self.pml_x = []   # same for Ex rows (top edges)
        if P <= 0:
            return
        top_c = np.arange(0, P)
        bot_c = np.arange(ny - P, ny)
        top_x = np.arange(1, P)                 # edge P is the interface (depth 0)
        bot_x = np.arange(ny - P + 1, ny)
        for rows, depth in ((top_c, P - top_c - 0.5), (bot_c, bot_c + 0.5 - (ny - P))):
            b, c, k = prof(depth)
            self.pml_c.append((rows, b[:, None], c[:, None], k[:, None],
                               np.zeros((len(rows), self.nx))))
        for rows, depth in ((top_x, (P - top_x).astype(float)),
                            (bot_x, (bot_x - (ny - P)).astype(float))):
            b, c, k = prof(depth)
            self.pml_x.append((rows, b[:, None], c[:, None], k[:, None],
                               np.zeros((len(rows), self.nx))))

    def step(self):
        dx, js = self.dx, self.js
        e_inc = self.inc.e_inc()                         # Ex_inc(edge js, n)
        self.inc.advance_h()
        h_inc = self.inc.h_inc()                         # Hz_inc(cell js, n+1/2)

        # Hz^{n-1/2} -> Hz^{n+1/2}  (Sec. 2.3, TEz Hz equation)
        ex_below = np.zeros_like(self.ex)
        ex_below[:-1] = self.ex[1:]                      # Ex[j+1]; Ex[ny] = 0
        d_ex = ex_below - self.ex                        # Ex[j+1] - Ex[j]
        if self.inc.kind != SOURCE_NONE:
            d_ex[js] -= e_inc                            # TF cell js sees total Ex[js]
        d_ey = np.roll(self.ey, -1, axis=1) - self.ey    # Ey[i+1] - Ey[i] (periodic)
        curl = (d_ey + d_ex) / dx
        for rows, b, c, k, psi in self.pml_c:
            psi *= b
            psi += c * d_ex[rows] / dx
            curl[rows] = d_ey[rows] / dx + d_ex[rows] / (k * dx) + psi
        self.hz = self.hz - self.ch_curl * curl

        tH = (self.n + 0.5) * self.dt
        self.dft["h_r"] += self.hz[self.jr] * np.exp(1j * self.omega * tH)
        self.dft["h_t"] += self.hz[self.jt] * np.exp(1j * self.omega * tH)

        # E^n -> E^{n+1}  (Sec. 2.3, TEz Ex and Ey equations)
        d_hz = self.hz[1:] - self.hz[:-1]                # Hz[j] - Hz[j-1], rows 1..ny-1
        if self.inc.kind != SOURCE_NONE:
            d_hz[js - 1] -= h_inc                        # SF edge js sees scattered Hz[js]
        term = d_hz / dx
        for rows, b, c, k, psi in self.pml_x:
            psi *= b
            psi += c * d_hz[rows - 1] / dx
            term[rows - 1] = d_hz[rows - 1] / (k * dx) + psi
        self.ex[1:] = self.cex[1:] * self.ex[1:] - self.cex_curl[1:] * term
        d_hz_x = self.hz - np.roll(self.hz, 1, axis=1)   # Hz[i] - Hz[i-1] (periodic)
        self.ey = self.cey * self.ey - self.cey_curl * d_hz_x / dx
        self.inc.advance_e()

        tE = (self.n + 1.0) * self.dt
        ph = np.exp(1j * self.omega * tE)
        self.dft["e_r"] += 0.5 * (self.ex[self.jr] + self.ex[self.jr + 1]) * ph
        self.dft["e_t"] += 0.5 * (self.ex[self.jt] + self.ex[self.jt + 1]) * ph
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

    def fields(self):
        return self.hz.copy(), self.ex.copy(), self.ey.copy()

    def fluxes(self):
        """Time-averaged Poynting fluxes (W/m per unit z-length): upward at
        r_row, downward at t_row, with P_down = 1/2 Re sum_i Ex~ conj(Hz~) dx."""
        d = self.dft
        p_r = -0.5 * np.real(np.sum(d["e_r"] * np.conj(d["h_r"]))) * self.dx
        p_t = 0.5 * np.real(np.sum(d["e_t"] * np.conj(d["h_t"]))) * self.dx
        return p_r, p_t


def empty_twin_tez(spec):
    """The empty-domain P-polarised run: one column of air."""
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
    return TEzOracle(s)


def run_rt_tez(spec, steps=None):
    """P-polarised R, T and A = 1 - R - T at lambda0 (Sec. 2.6), normalised
    by the empty-domain run scaled to nx columns."""
    steps = spec.steps if steps is None else steps
    leaf = TEzOracle(spec).run(steps)
    twin = empty_twin_tez(spec).run(steps)
    p_up, p_down = leaf.fluxes()
    _, p0 = twin.fluxes()
    p_inc = p0 * spec.nx
    R, T = p_up / p_inc, p_down / p_inc
    return dict(R=R, T=T, A=1.0 - R - T, p_up=p_up, p_down=p_down, p_inc=p_inc,
                leaf=leaf, twin=twin)


def unpolarized(rt_s, rt_p):
    """Unpolarised illumination (Sec. 2.1): the S (TMz) and P (TEz) runs are
    independent and carry equal incident power, so R, T and A of natural
    light are the means of the two polarisations."""
    return {k: 0.5 * (rt_s[k] + rt_p[k]) for k in ("R", "T", "A")}
