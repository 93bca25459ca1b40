"""FP64 discrete adjoint of the TMz FDTD objective (test infrastructure).

The forward map is the oracle's leapfrog loop (fdtd_tmz.TMzOracle) with
per-cell eps_r and sigma; the objective is J = wR R + wT T with R and T the
Poynting-flux ratios of Sec. 2.6 (the incident power comes from the empty
domain and does not depend on the cell parameters). The gradient is obtained
by running the exact transpose of every update of the forward step in
reverse order (reverse-mode differentiation of the discrete recursion):

  forward step n:  psi_e <- b psi_e + c d_hx/dx           (CPML rows)
                   Ez    <- Ce Ez + Cc curl,  curl = (d_hy + d_hx/kappa)/dx + psi_e
                   DFT of Ez at the monitor rows
                   psi_h <- b psi_h + c d_ez/dx            (CPML rows)
                   Hx    <- Hx + dt/mu0 (d_ez/(kappa dx) + psi_h),  Hy <- Hy + dt/mu0 d_ezx/dx
                   DFT of the row-averaged Hx
  reverse step n (adjoint variables lE, lX, lY and the CPML carries):
                   monitor sources, transpose of the H updates, monitor
                   source of E, then gCe += lE Ez^{n-1/2}, gCc += lE curl^n
                   and the transpose of the E update.

Ce = (1-b)/(1+b) and Cc = dt/(eps0 eps_r (1+b)), b = sigma dt/(2 eps0 eps_r)
(Sec. 2.3) are then differentiated in closed form, and (eps_r, sigma) in
terms of (n, kappa) (Sec. 2.2) for the per-label gradient.

Pins: tests/test_oracle_adjoint.py (dot-product transpose test of the step
operator, central finite differences on every cell of a small grid).
"""
from __future__ import annotations

import math

import numpy as np

from .fdtd_tmz import EPS0, TMzOracle, empty_twin


def reverse_step(sim, adj, n, src=None):
    """Transpose of forward step n applied to the adjoint state `adj`
    (dict with lE, lX, lY and lists mE, mH of CPML carries, in place).
    `src` holds the monitor sources (None for the bare linear operator).
    Returns the adjoint of Ez^{n+1/2} seen by the Ez update (for gradients)."""
    dx, dtmu = sim.dx, sim.ch_curl
    lE, lX, lY = adj["lE"], adj["lX"], adj["lY"]
    if src is not None:
        kR, kT, er, et = src["kR"], src["kT"], src["e_r"], src["e_t"]
        ph = np.exp(1j * sim.omega * (n + 1.0) * sim.dt)
        gr = 0.5 * kR * np.real(er * np.conj(ph))
        gt = 0.5 * kT * np.real(et * np.conj(ph))
        lX[sim.jr] += gr
        lX[sim.jr + 1] += gr
        lX[sim.jt] += gt
        lX[sim.jt + 1] += gt
    # transpose of Hy <- Hy + dtmu (Ez[i] - Ez[i-1])/dx
    gy = dtmu * lY / dx
    lE += gy - np.roll(gy, -1, axis=1)
    # transpose of Hx[1:] <- Hx[1:] + dtmu term(d_ez), d_ez = Ez[j] - Ez[j-1]
    dbar = dtmu * lX[1:] / dx                      # adjoint of d_ez (rows 1..ny-1)
    for q, (rows, b, c, k, _psi) in enumerate(sim.pml_h):
        nu = dtmu * lX[rows] + adj["mH"][q]        # total adjoint of psi_h^{n+1}
        dbar[rows - 1] = dtmu * lX[rows] / (k * dx) + c * nu / dx
        adj["mH"][q] = b * nu
    lE[1:] += dbar
    lE[:-1] -= dbar
    if src is not None:
        kR, kT, hr, ht = src["kR"], src["kT"], src["h_r"], src["h_t"]
        pe = np.exp(1j * sim.omega * (n + 0.5) * sim.dt)
        lE[sim.jr] += kR * np.real(hr * np.conj(pe))
        lE[sim.jt] += kT * np.real(ht * np.conj(pe))
    ebar = lE.copy()
    # transpose of Ez <- Ce Ez + Cc curl
    cbar = sim.ce_curl * ebar                      # adjoint of curl
    ghy = cbar / dx                                # adjoint of d_hy
    ghx = cbar / dx                                # adjoint of d_hx
    for q, (rows, b, c, k, _psi) in enumerate(sim.pml_e):
        rho = cbar[rows] + adj["mE"][q]            # total adjoint of psi_e^n
        ghx[rows] = cbar[rows] / (k * dx) + c * rho / dx
        adj["mE"][q] = b * rho
    # d_hy = Hy[i+1] - Hy[i];  d_hx = Hx[j+1] - Hx[j]
    lY += np.roll(ghy, 1, axis=1) - ghy
    lX[1:] += ghx[:-1]
    lX -= ghx
    adj["lE"] = sim.ce * ebar
    return ebar


def new_adjoint_state(sim):
    z = np.zeros((sim.ny, sim.nx))
    return {"lE": z.copy(), "lX": z.copy(), "lY": z.copy(),
            "mE": [np.zeros_like(blk[4]) for blk in sim.pml_e],
            "mH": [np.zeros_like(blk[4]) for blk in sim.pml_h]}


def coefficient_derivatives(eps_r, sigma, dt):
    """d(Ce)/d(eps_r), d(Ce)/d(sigma), d(Cc)/d(eps_r), d(Cc)/d(sigma) for
    Ce = (1-b)/(1+b), Cc = dt/(eps0 eps_r (1+b)), b = sigma dt/(2 eps0 eps_r)."""
    b = sigma * dt / (2.0 * EPS0 * eps_r)
    q = (1.0 + b) ** 2
    dce_de = 2.0 * b / (eps_r * q)
    dce_ds = -dt / (EPS0 * eps_r * q)
    dcc_de = -dt / (EPS0 * eps_r ** 2 * q)
    dcc_ds = -dt * dt / (2.0 * EPS0 ** 2 * eps_r ** 2 * q)
    return dce_de, dce_ds, dcc_de, dcc_ds


def objective_and_gradient(spec, steps, wR=1.0, wT=0.0, eps_r=None, sigma=None):
    """J = wR R + wT T after `steps` steps and dJ/d(eps_r), dJ/d(sigma) per
    cell; with labels, also dJ/dn and dJ/dkappa per label (Sec. 2.2)."""
    sim = TMzOracle(spec, eps_r=eps_r, sigma=sigma)
    sim.tape = []
    sim.run(steps)
    tape = sim.tape
    twin = empty_twin(spec).run(steps)
    p_inc = twin.fluxes()[1] * spec.nx
    p_up, p_down = sim.fluxes()
    R, T = p_up / p_inc, p_down / p_inc
    J = wR * R + wT * T
    d = sim.dft
    src = {"kR": wR * 0.5 * sim.dx / p_inc, "kT": -wT * 0.5 * sim.dx / p_inc,
           "e_r": d["e_r"], "e_t": d["e_t"], "h_r": d["h_r"], "h_t": d["h_t"]}
    adj = new_adjoint_state(sim)
    g_ce = np.zeros((sim.ny, sim.nx))
    g_cc = np.zeros((sim.ny, sim.nx))
    for n in range(int(steps) - 1, -1, -1):
        e_prev, curl = tape[n]
        ebar = reverse_step(sim, adj, n, src)
        g_ce += ebar * e_prev
        g_cc += ebar * curl
    dce_de, dce_ds, dcc_de, dcc_ds = coefficient_derivatives(sim.eps_r, sim.sigma, sim.dt)
    g_eps = g_ce * dce_de + g_cc * dcc_de
    g_sig = g_ce * dce_ds + g_cc * dcc_ds
    out = {"J": J, "R": R, "T": T, "g_eps": g_eps, "g_sigma": g_sig}
    if eps_r is None:
        mats = np.asarray(spec.materials, dtype=np.float64)
        lab = np.asarray(spec.labels)
        n_l, k_l = mats[:, 0], mats[:, 1]
        w = sim.omega * EPS0
        g_n = np.zeros(len(mats))
        g_k = np.zeros(len(mats))
        for l in range(len(mats)):
            m = lab == l
            # eps_r = n^2 - k^2, sigma = 2 w eps0 n k
            g_n[l] = np.sum(g_eps[m] * 2.0 * n_l[l] + g_sig[m] * 2.0 * w * k_l[l])
            g_k[l] = np.sum(-g_eps[m] * 2.0 * k_l[l] + g_sig[m] * 2.0 * w * n_l[l])
        out["g_n"], out["g_k"] = g_n, g_k
    return out


def incident_power(spec, steps):
    """P_inc of the empty-domain run (independent of the cell parameters)."""
    return empty_twin(spec).run(steps).fluxes()[1] * spec.nx


def objective(spec, steps, wR=1.0, wT=0.0, eps_r=None, sigma=None, p_inc=None):
    """J alone (the forward half of objective_and_gradient)."""
    sim = TMzOracle(spec, eps_r=eps_r, sigma=sigma).run(steps)
    if p_inc is None:
        p_inc = incident_power(spec, steps)
    p_up, p_down = sim.fluxes()
    return wR * p_up / p_inc + wT * p_down / p_inc


def maps_from_labels(spec):
    """Per-cell eps_r, sigma of a labelled spec at its wavelength."""
    from .fdtd_tmz import C0, eps_sigma
    mats = np.asarray(spec.materials, dtype=np.float64)
    lab = np.asarray(spec.labels)
    return eps_sigma(mats[lab, 0], mats[lab, 1], 2.0 * math.pi * C0 / spec.lambda0)
