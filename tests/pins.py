"""Independent closed forms that pin the FP64 oracle (test helpers).

Nothing here runs a time-stepping loop. The frequency-domain lattice solver
works on the steady-state equations of the Yee scheme at one frequency, and
the continuum formulas are the textbook transfer matrices (Airy / Fresnel).
"""
from __future__ import annotations

import math

import numpy as np

C0 = 299_792_458.0
MU0 = 4.0e-7 * math.pi
EPS0 = 1.0 / (MU0 * C0 * C0)


def lattice_wavenumber(omega, dx, dt, n=1.0, kappa=0.0):
    """Wavenumber of a plane wave on the 1D Yee lattice in a uniform medium.

    Steady state at e^{-i w t} of the discrete updates gives, with
    theta = w dt/2 and w~ = 2 sin(theta)/dt,
      (-i w~ eps0 eps_r + sigma cos(theta)) E_j = (H_{j+1} - H_j)/dx,
      -i w~ mu0 H_j = (E_j - E_{j-1})/dx,
    so 4 sin^2(k dx/2) = dx^2 w~ mu0 (w~ eps0 eps_r + i sigma cos(theta)).
    The root with Im k >= 0, Re k >= 0 (wave moving to +s) is returned.
    """
    theta = omega * dt / 2.0
    wt = 2.0 * math.sin(theta) / dt
    eps_c = (n + 1j * kappa) ** 2          # eps_r + i sigma/(omega eps0)
    eps_r, sig = eps_c.real, eps_c.imag * omega * EPS0
    rhs = dx * dx * wt * MU0 * (wt * EPS0 * eps_r + 1j * sig * math.cos(theta))
    s = np.sqrt(rhs + 0j) / 2.0            # sin(k dx/2)
    k = 2.0 * np.arcsin(s) / dx
    if k.imag < 0 or (abs(k.imag) < 1e-300 and k.real < 0):
        k = -k
    return complex(k)


def lattice_stack_rt(omega, dx, dt, row_index):
    """R and T of an x-uniform stack on the Yee lattice (exact discrete
    steady state). row_index: list of complex indices n + i kappa per Ez row;
    the first row must be air. Below the last row the medium of the last row
    continues (a half-space when it is not air; T is then None).

    The recurrences are marched upward from a pure outgoing (downward)
    lattice wave below the stack and the field above it is split into its
    incident and reflected lattice waves.
    """
    theta = omega * dt / 2.0
    wt = 2.0 * math.sin(theta) / dt
    N = len(row_index)
    # coefficients of  a_j E_j = H_{j+1} - H_j  and  g H_j = E_j - E_{j-1}
    a = np.empty(N, dtype=np.complex128)
    for j, nk in enumerate(row_index):
        eps_c = complex(nk) ** 2
        eps_r, sig = eps_c.real, eps_c.imag * omega * EPS0
        a[j] = dx * (-1j * wt * EPS0 * eps_r + sig * math.cos(theta))
    g = -1j * wt * MU0 * dx
    k0 = lattice_wavenumber(omega, dx, dt)
    s0 = 2j * math.sin(k0.real * dx / 2.0)
    nb = complex(row_index[-1])
    kb = lattice_wavenumber(omega, dx, dt, nb.real, nb.imag)
    sb = 2j * np.sin(kb * dx / 2.0)
    # below the stack: E_j = e^{i k (j+1/2) dx}, H_j = (s/g) e^{i k j dx}
    jb = N - 1
    E = np.exp(1j * kb * (jb + 0.5) * dx)
    H_next = (sb / g) * np.exp(1j * kb * (jb + 1) * dx)
    t_amp = 1.0
    Ej = E
    for j in range(jb, 0, -1):
        Hj = H_next - a[j] * Ej
        Ejm1 = Ej - g * Hj
        H_next, Ej = Hj, Ejm1
    # now Ej = E_0 and H_next = H_1; air at row 0 and 1:
    # E_0 = A e^{i k dx/2} + B e^{-i k dx/2};  H_1 = (s0/g)(A e^{i k dx} - B e^{-i k dx})
    M = np.array([[np.exp(1j * k0 * 0.5 * dx), np.exp(-1j * k0 * 0.5 * dx)],
                  [(s0 / g) * np.exp(1j * k0 * dx), -(s0 / g) * np.exp(-1j * k0 * dx)]])
    A, B = np.linalg.solve(M, np.array([Ej, H_next]))
    T = abs(t_amp / A) ** 2 if nb == 1.0 else None
    return abs(B / A) ** 2, T


def continuum_stack_rt(lambda0, layers):
    """Textbook normal-incidence transfer matrix for air | layers | air.
    layers: [(thickness_m, n + i kappa), ...] (e^{-i w t} convention)."""
    k0 = 2.0 * math.pi / lambda0
    M = np.eye(2, dtype=np.complex128)
    for d, nc in layers:
        delta = k0 * nc * d
        Y = nc
        M = M @ np.array([[np.cos(delta), -1j * np.sin(delta) / Y],
                          [-1j * Y * np.sin(delta), np.cos(delta)]])
    n_in = n_out = 1.0
    den = n_in * M[0, 0] + n_in * n_out * M[0, 1] + M[1, 0] + n_out * M[1, 1]
    r = (n_in * M[0, 0] + n_in * n_out * M[0, 1] - M[1, 0] - n_out * M[1, 1]) / den
    t = 2.0 * n_in / den
    return abs(r) ** 2, abs(t) ** 2 * (n_out / n_in)


def rows_to_index(ny, layers):
    """Per-row complex index for an x-uniform stack: layers = [(r0, r1, nk)]."""
    idx = [1.0 + 0j] * ny
    for r0, r1, nk in layers:
        for j in range(r0, r1):
            idx[j] = nk
    return idx


def lattice_stack_rt_tez(omega, dx, dt, row_index):
    """R and T of an x-uniform stack on the P-polarised (TEz) Yee lattice:
    Hz at cell centres, Ex on the horizontal edges, each edge taking the
    mean complex permittivity of the two cells it separates. Steady state
    at e^{-i w t} (theta = w dt/2, w~ = 2 sin(theta)/dt):
      -i w~ mu0 Hz_j = -(Ex_{j+1} - Ex_j)/dx,
      (-i w~ eps0 eps_e + sigma_e cos(theta)) Ex_j = -(Hz_j - Hz_{j-1})/dx.
    row_index as for lattice_stack_rt (rows 0 and 1 air; the last row's
    medium continues below, T is None when it is not air).
    """
    theta = omega * dt / 2.0
    wt = 2.0 * math.sin(theta) / dt
    N = len(row_index)
    eps_c = np.array([complex(nk) ** 2 for nk in row_index])
    # edge j separates rows j-1 and j (edges 1..N-1); the mean of eps_r and
    # sigma is the mean of the complex permittivity
    a = np.zeros(N + 1, dtype=np.complex128)
    for j in range(1, N):
        e = 0.5 * (eps_c[j - 1] + eps_c[j])
        a[j] = dx * (-1j * wt * EPS0 * e.real + e.imag * omega * EPS0 * math.cos(theta))
    g = -1j * wt * MU0 * dx
    k0 = lattice_wavenumber(omega, dx, dt)
    s0 = 2j * math.sin(k0.real * dx / 2.0)
    nb = complex(row_index[-1])
    kb = lattice_wavenumber(omega, dx, dt, nb.real, nb.imag)
    sb = 2j * np.sin(kb * dx / 2.0)
    # outgoing wave in the bottom medium: Ex_j = e^{i k j dx},
    # Hz_j = -(s/g) e^{i k (j+1/2) dx}; it holds down from edge N-1 and
    # centre N-1, whose equations involve no averaged edge
    Ex = np.exp(1j * kb * (N - 1) * dx)
    Hz = -(sb / g) * np.exp(1j * kb * (N - 0.5) * dx)
    for j in range(N - 1, 1, -1):
        Hz = Hz + a[j] * Ex            # Hz_{j-1} from the edge-j equation
        Ex = Ex + g * Hz               # Ex_{j-1} from the centre-(j-1) equation
    Hz0 = Hz + a[1] * Ex               # Hz_0; Ex now holds Ex_1
    # air: Ex_1 = A e^{i k dx} + B e^{-i k dx},
    #      Hz_0 = -(s0/g) (A e^{i k dx/2} - B e^{-i k dx/2})
    M = np.array([[np.exp(1j * k0 * dx), np.exp(-1j * k0 * dx)],
                  [-(s0 / g) * np.exp(0.5j * k0 * dx), (s0 / g) * np.exp(-0.5j * k0 * dx)]])
    A, B = np.linalg.solve(M, np.array([Ex, Hz0]))
    T = abs(1.0 / A) ** 2 if nb == 1.0 else None
    return abs(B / A) ** 2, T
