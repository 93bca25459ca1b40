"""Bloch-order decomposition of the monitor lines (Sec. 2.6), FP64.

TEST INFRASTRUCTURE: used only by tests/ to check the CUDA library.

The fields are periodic in x with period L = nx dx, so the DFT of a monitor
line expands as E(x) = sum_m E_m exp(i k_{x,m} x), k_{x,m} = 2 pi m / L, with
E_m = (1/nx) sum_i E_i exp(-2 pi i m i / nx). An order propagates when its
longitudinal wavenumber is real. On the lattice that wavenumber follows the
2D dispersion relation
    sin^2(k_y dx/2) = sin^2(w dt/2) / S^2 - sin^2(k_x dx/2),
which tends to k_y^2 = k0^2 - k_x^2 as dx -> 0.

Sec. 2.6 sums |E_m|^2 / |E_inc,0|^2 over the propagating orders (E = Ez for
S, Ex for P). That ratio is the power of order m only for m = 0: an oblique
order carries a power proportional to |E_m|^2 k_y/k0 (Ez) or
|E_m|^2 k0/k_y (Ex). On the lattice, with the DFT time stamps of the
monitors and the row-averaged edge field, the exact factors are
    w_m = sin(k_{y,m} dx) / sin(k_{y,0} dx)      (S: Ez amplitudes),
    w_m = sin(k_{y,0} dx) / sin(k_{y,m} dx)      (P: Ex amplitudes),
because a one-way lattice wave has averaged-edge / centre phasor ratio
-S sin(k_y dx) / (2 sin(w dt/2)). Both the paper's sums and the corrected
ones are returned, with the exact split of the Poynting flux by order
(Parseval: sum_i E_i conj(H_i) = nx sum_m E_m conj(H_m)).
"""
from __future__ import annotations

import math

import numpy as np

from .fdtd_tmz import C0


def lattice_ky(m, nx, dx, dt, omega):
    """k_y dx of order m on the lattice (nan where the order is evanescent)."""
    S = C0 * dt / dx
    s2 = math.sin(omega * dt / 2.0) ** 2 / (S * S) - np.sin(np.pi * np.asarray(m) / nx) ** 2
    s2 = np.asarray(s2, dtype=np.float64)
    out = np.full(s2.shape, np.nan)
    ok = (s2 > 0.0) & (s2 <= 1.0)
    out[ok] = 2.0 * np.arcsin(np.sqrt(s2[ok]))
    return out


def propagating_orders(nx, dx, dt, omega):
    """Largest M such that every |m| <= M propagates on the lattice."""
    M = 0
    while M + 1 < nx // 2 + 1 and np.isfinite(lattice_ky(M + 1, nx, dx, dt, omega)):
        M += 1
    return M


def bloch_orders(leaf, twin, m_max=None):
    """Per-order reflectance and transmittance of a finished run.

    leaf, twin: a TMzOracle / TEzOracle run and its empty-domain run (same
    polarisation). Orders m = -m_max..m_max (default: all propagating ones).
    Returns a dict of arrays over m: m, ky (k_y dx, nan if evanescent), w
    (obliquity factor, 0 if evanescent), R_flux / T_flux (order m's share of
    the Poynting fluxes over P_inc), R_paper / T_paper (|E_m|^2/|E_inc,0|^2),
    R_corr / T_corr (w |E_m|^2/|E_inc,0|^2), and the totals R, T of the run.
    """
    from .fdtd_tez import TEzOracle
    p_te = isinstance(leaf, TEzOracle)
    nx, dx, dt = leaf.nx, leaf.dx, leaf.dt
    if m_max is None:
        m_max = propagating_orders(nx, dx, dt, leaf.omega)
    m = np.arange(-m_max, m_max + 1)
    d, dt_ = leaf.dft, twin.dft
    if p_te:
        # Poynting pair (Ex, Hz); the paper's E is Ex (row-averaged edges)
        pe_r, ph_r, pe_t, ph_t = d["e_r"], d["h_r"], d["e_t"], d["h_t"]
        sign_r, sign_t = -1.0, 1.0          # P_up = -1/2 Re sum Ex Hz*, P_down = +...
        e_inc = dt_["e_t"][0]
        p_inc = 0.5 * np.real(dt_["e_t"][0] * np.conj(dt_["h_t"][0])) * dx * nx
    else:
        pe_r, ph_r, pe_t, ph_t = d["e_r"], d["h_r"], d["e_t"], d["h_t"]
        sign_r, sign_t = 1.0, -1.0          # P_up = +1/2 Re sum Ez Hx*, P_down = -...
        e_inc = dt_["e_t"][0]
        p_inc = -0.5 * np.real(dt_["e_t"][0] * np.conj(dt_["h_t"][0])) * dx * nx

    def orders(line):
        f = np.fft.fft(line) / nx                    # index m mod nx
        return f[m % nx]

    Er, Hr, Et, Ht = orders(pe_r), orders(ph_r), orders(pe_t), orders(ph_t)
    R_flux = sign_r * 0.5 * np.real(Er * np.conj(Hr)) * nx * dx / p_inc
    T_flux = sign_t * 0.5 * np.real(Et * np.conj(Ht)) * nx * dx / p_inc
    ky = lattice_ky(m, nx, dx, dt, leaf.omega)
    ky0 = lattice_ky(0, nx, dx, dt, leaf.omega)
    prop = np.isfinite(ky)
    w = np.zeros(len(m))
    if p_te:
        w[prop] = np.sin(ky0) / np.sin(ky[prop])
    else:
        w[prop] = np.sin(ky[prop]) / np.sin(ky0)
    R_paper = np.abs(Er) ** 2 / abs(e_inc) ** 2
    T_paper = np.abs(Et) ** 2 / abs(e_inc) ** 2
    p_up, p_down = leaf.fluxes()
    return dict(m=m, ky=ky, w=w, R_flux=R_flux, T_flux=T_flux, R_paper=R_paper,
                T_paper=T_paper, R_corr=w * R_paper, T_corr=w * T_paper,
                R=p_up / p_inc, T=p_down / p_inc)
