"""Pins of the FP64 P-polarisation (TEz) oracle. Each right-hand side comes
from mathematics the oracle does not execute: the steady-state lattice
recurrences of x-uniform stacks solved in the frequency domain, textbook
transfer matrices, the 2D lattice dispersion relation of a cavity mode, the
E/H duality of Maxwell's equations in air, exact mirror symmetry and the
energy conservation of a lossless structure."""
import math

import numpy as np
import pytest

from fdtd_inputs import config_c1, courant_dt
from fdtd_inputs.geometry import cylinder_array_labels, stack_labels
from oracle import C0, ETA0, TMzOracle, run_rt
from oracle.fdtd_tez import (TEzOracle, edge_materials, empty_twin_tez, run_rt_tez,
                             unpolarized)
import pins

LAM = 550e-9
W0 = 2 * math.pi * C0 / LAM
C1_LAYERS = [(40, 90, 1), (90, 215, 2)]


def _spec_1d(ny=256, layers=(), steps=4000, nx=1, **kw):
    base = config_c1(nx=nx, steps=steps)
    lab = stack_labels(nx, ny, list(layers))
    return base.with_(ny=ny, labels=lab, **kw)


# -- x-uniform stacks: the exact TEz lattice -------------------------------------------

def test_tez_slab_rt_matches_discrete_lattice():
    spec = _spec_1d(layers=C1_LAYERS, steps=8000)
    r = run_rt_tez(spec)
    idx = pins.rows_to_index(256, [(40, 90, 1.45), (90, 215, 1.42 + 1e-3j)])
    R, T = pins.lattice_stack_rt_tez(W0, spec.dx, spec.dt, idx)
    assert abs(r["R"] - R) < 1e-5 and abs(r["T"] - T) < 1e-5


def test_tez_lossless_slab_conserves_energy():
    spec = _spec_1d(layers=C1_LAYERS, steps=8000)
    spec = spec.with_(materials=np.array([[1.0, 0.0], [1.45, 0.0], [1.42, 0.0]]))
    r = run_rt_tez(spec)
    assert abs(r["R"] + r["T"] - 1.0) < 1e-5
    R, _ = pins.lattice_stack_rt_tez(W0, spec.dx, spec.dt,
                                     pins.rows_to_index(256, [(40, 90, 1.45), (90, 215, 1.42)]))
    assert abs(r["R"] - R) < 1e-5


def test_tez_beer_lambert_index_matched_layer():
    spec = _spec_1d(layers=[(90, 215, 1)], steps=6000)
    spec = spec.with_(materials=np.array([[1.0, 0.0], [1.0, 1e-3]]))
    r = run_rt_tez(spec)
    assert abs(r["T"] - math.exp(-4 * math.pi * 1e-3 * 2.5e-6 / LAM)) < 3e-4
    R, T = pins.lattice_stack_rt_tez(W0, spec.dx, spec.dt,
                                     pins.rows_to_index(256, [(90, 215, 1.0 + 1e-3j)]))
    assert abs(r["T"] - T) < 1e-5 and abs(r["R"] - R) < 1e-6


def test_tez_fresnel_half_space():
    ny = 256
    spec = _spec_1d(ny=ny, layers=[(120, ny, 1)], steps=6000)
    spec = spec.with_(materials=np.array([[1.0, 0.0], [1.45, 0.0]]))
    r = run_rt_tez(spec)
    R_lat, _ = pins.lattice_stack_rt_tez(W0, spec.dx, spec.dt,
                                         pins.rows_to_index(200, [(100, 200, 1.45)]))
    assert abs(r["R"] - R_lat) < 1e-5
    assert abs(r["R"] - ((1.45 - 1) / 2.45) ** 2) < 2e-3


def test_tez_lattice_pin_tends_to_continuum():
    # the pin itself: second-order convergence to the Airy value, and the
    # half-space to Fresnel (the averaged edge sits on the interface)
    errs, errs_if = [], []
    Rc, Tc = pins.continuum_stack_rt(LAM, [(1e-6, 1.45), (2.5e-6, 1.42 + 1e-3j)])
    for d in (20e-9, 10e-9, 5e-9):
        dt = 0.5 * d / C0
        n1, n2 = int(round(1e-6 / d)), int(round(2.5e-6 / d))
        idx = pins.rows_to_index(n1 + n2 + 20, [(10, 10 + n1, 1.45),
                                                (10 + n1, 10 + n1 + n2, 1.42 + 1e-3j)])
        R, T = pins.lattice_stack_rt_tez(W0, d, dt, idx)
        errs.append(abs(R - Rc) + abs(T - Tc))
        Ri, _ = pins.lattice_stack_rt_tez(W0, d, dt, pins.rows_to_index(40, [(20, 40, 1.45)]))
        errs_if.append(abs(Ri - ((1.45 - 1) / 2.45) ** 2))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
    assert errs_if[0] / errs_if[1] > 3.5 and errs_if[1] / errs_if[2] > 3.5


@pytest.mark.parametrize("kappa_max", [1.0, 4.0])
def test_tez_cpml_reflection_below_1e_minus_4(kappa_max):
    spec = _spec_1d(layers=[], steps=8000, pml_kappa_max=kappa_max)
    p_up, p_down = empty_twin_tez(spec).run(8000).fluxes()
    assert p_down > 0 and p_up / p_down < 1e-9


def test_tez_vacuum_dispersion_and_zero_sf_leakage():
    ny, steps = 2000, 3600
    spec = _spec_1d(ny=ny, steps=steps, r_row=300, t_row=310)
    sim = TEzOracle(spec)
    leak, peak = 0.0, 0.0
    for _ in range(steps):
        sim.step()
        leak = max(leak, np.abs(sim.hz[: spec.tfsf_row]).max() * ETA0,
                   np.abs(sim.ex[: spec.tfsf_row + 1]).max())
        peak = max(peak, np.abs(sim.ex).max())
    assert leak <= 1e-12 * peak
    k = 2.0 / spec.dx * math.asin(math.sin(W0 * spec.dt / 2) / spec.courant)
    ratio = sim.dft["h_t"][0] / sim.dft["h_r"][0]
    assert abs(ratio - np.exp(1j * k * 10 * spec.dx)) < 1e-8
    # a one-way lattice wave: the row-averaged Ex phasor (time stamps n+1) is
    # +cos(k dx/2) eta0 times the Hz phasor (time stamps n+1/2)
    for row in ("r", "t"):
        eh = sim.dft["e_" + row][0] / (ETA0 * sim.dft["h_" + row][0])
        assert abs(eh - math.cos(k * spec.dx / 2)) < 1e-9


# -- duality, cavity modes, symmetry, conservation ------------------------------------

def test_duality_with_tmz_in_air():
    # In air, (E, H) -> (eta0 H, -E / eta0) maps TMz onto TEz: eta0 Hz = Ez and
    # Ex = -eta0 Hx for the same incident waveform, CPML and monitors.
    spec = _spec_1d(layers=[], steps=900, nx=3)
    tm = TMzOracle(spec).run(900)
    te = TEzOracle(spec).run(900)
    scale = np.abs(tm.ez).max()
    assert scale > 0.1
    assert np.abs(ETA0 * te.hz - tm.ez).max() <= 1e-12 * scale
    assert np.abs(te.ex + ETA0 * tm.hx).max() <= 1e-12 * scale
    assert np.abs(te.ey).max() == 0.0
    p_tm, p_te = tm.fluxes(), te.fluxes()
    assert abs(p_te[1] - p_tm[1]) <= 1e-12 * abs(p_tm[1]) and p_tm[1] > 0


def _cavity(nx, ny, courant, n=1.0):
    base = config_c1(nx=nx, steps=1)
    return base.with_(ny=ny, nx=nx, dt=courant_dt(base.dx, courant),
                      labels=np.zeros((ny, nx), np.uint8),
                      materials=np.array([[n, 0.0]]), pml_cells=0,
                      source_kind=2, tfsf_row=2, r_row=1, t_row=ny - 3)


@pytest.mark.parametrize("mx,my,courant,n", [(3, 2, 0.5, 1.0), (1, 5, 0.5, 1.5),
                                             (12, 9, 0.7071, 1.0), (4, 0, 0.6, 1.5)])
def test_tez_cavity_eigenmode_closed_form(mx, my, courant, n):
    # Periodic x, Ex = 0 on the top and bottom walls: Hz = cos(kx x) cos(ky s)
    # oscillates at the 2D lattice frequency
    # sin^2(w dt/2) = (S^2 / n^2) (sin^2(kx dx/2) + sin^2(ky dx/2)).
    nx, ny = 24, 18
    spec = _cavity(nx, ny, courant, n)
    dx, dt = spec.dx, spec.dt
    S = C0 * dt / dx
    kx = 2 * math.pi * mx / (nx * dx)
    ky = math.pi * my / (ny * dx)
    s2 = (S / n) ** 2 * (math.sin(kx * dx / 2) ** 2 + math.sin(ky * dx / 2) ** 2)
    w = 2.0 * math.asin(math.sqrt(s2)) / dt
    i, j = np.arange(nx), np.arange(ny)
    shape = np.outer(np.cos(ky * (j + 0.5) * dx), np.cos(kx * (i + 0.5) * dx + 0.3))
    sim = TEzOracle(spec)
    sim.hz = math.cos(w * dt / 2) * shape        # Hz^{-1/2}; E^0 = 0
    for step in range(400):
        sim.step()
        expect = math.cos(w * (step + 0.5) * dt) * shape
        assert np.abs(sim.hz - expect).max() < 1e-11
    assert np.abs(sim.ex[0]).max() == 0.0


def test_tez_lossy_mode_decays_with_det_ce():
    # A ky = 0 mode in a uniform lossy medium evolves by a 2x2 map per step
    # (a shear for Hz, a scaled shear for Ey) whose determinant is C_e, so the
    # mode's eigenvalues have modulus sqrt(C_e) = exp(-sigma dt/(2 eps)) + O(b^3).
    nx, ny = 24, 6
    spec = _cavity(nx, ny, 0.5, 1.3).with_(materials=np.array([[1.3, 0.02]]))
    dt = spec.dt
    sim = TEzOracle(spec)
    kx = 2 * math.pi * 2 / (nx * spec.dx)
    xc = (np.arange(nx) + 0.5) * spec.dx
    xe = np.arange(nx) * spec.dx
    sim.hz = np.tile(np.cos(kx * xc), (ny, 1))
    states = []
    for _ in range(3):
        # mode amplitudes: Hz on cos(kx x), Ey on sin(kx x) (Ey at the edges)
        states.append([sim.hz[0] @ np.cos(kx * xc), sim.ey[0] @ np.sin(kx * xe)])
        sim.step()
    s = np.array(states).T
    M = s[:, 1:] @ np.linalg.inv(s[:, :2])
    ce = sim.cey[0, 0]
    eps_r, sig = 1.3 ** 2 - 0.02 ** 2, 2 * W0 * 8.8541878128e-12 * 1.3 * 0.02
    b = sig * dt / (2 * 8.8541878128e-12 * eps_r)
    assert abs(np.linalg.det(M) - ce) < 1e-12
    assert abs(ce - (1 - b) / (1 + b)) < 1e-15
    assert abs(math.sqrt(ce) - math.exp(-b)) < b ** 3


def test_edge_materials_are_cell_means():
    eps = np.array([[1.0, 2.0, 4.0], [3.0, 5.0, 7.0]])
    sig = np.array([[0.0, 1.0, 2.0], [4.0, 8.0, 16.0]])
    ex_e, ex_s, ey_e, ey_s = edge_materials(eps, sig)
    assert np.array_equal(ex_e[1], [2.0, 3.5, 5.5]) and np.array_equal(ex_s[1], [2.0, 4.5, 9.0])
    assert np.array_equal(ey_e[0], [2.5, 1.5, 3.0]) and np.array_equal(ey_s[1], [10.0, 6.0, 12.0])


def _cylinders(nx=24, steps=5000, lossless=True):
    lab = stack_labels(nx, 256, [(40, 90, 1), (90, 215, 2)])
    disc = cylinder_array_labels(nx, 60, 0.375 * nx)
    lab[120:180][disc == 1] = 3
    mats = np.array([[1.0, 0.0], [1.45, 0.0], [1.42, 0.0 if lossless else 1e-3], [2.0, 0.0]])
    return config_c1(nx=nx, steps=steps).with_(labels=lab, materials=mats)


def test_tez_mirror_symmetry_is_exact():
    spec = _cylinders(steps=700, lossless=False)
    assert np.array_equal(spec.labels, spec.labels[:, ::-1])
    sim = TEzOracle(spec).run(700)
    hz, ex, ey = sim.fields()
    assert np.abs(ex).max() > 0.1 and np.abs(ey).max() > 1e-4
    assert np.array_equal(hz, hz[:, ::-1]) and np.array_equal(ex, ex[:, ::-1])
    # Ey on edge i mirrors to edge (nx - i) mod nx with a sign change
    assert np.array_equal(ey, -np.roll(ey[:, ::-1], 1, axis=1))


def test_tez_lossless_2d_structure_conserves_energy():
    # period 240 nm < 550 nm / 2: every diffraction order but the zeroth is
    # evanescent even in the n = 2 cylinders, so no guided mode of the slab
    # is excited and the fluxes of the lossless structure balance once the
    # pulse has left (a 480 nm period rings in slab modes for >> 6000 steps)
    r = run_rt_tez(_cylinders(nx=12, steps=6000))
    assert abs(r["R"] + r["T"] - 1.0) < 1e-5
    assert r["R"] > 0.01 and np.abs(r["leaf"].ey).max() >= 0.0


def test_unpolarized_is_the_mean_of_both_runs():
    spec = _spec_1d(layers=C1_LAYERS, steps=8000)
    s, p = run_rt(spec), run_rt_tez(spec)
    u = unpolarized(s, p)
    for k in ("R", "T", "A"):
        assert u[k] == 0.5 * (s[k] + p[k])
    assert abs(u["A"] - (1.0 - u["R"] - u["T"])) < 1e-15
    assert empty_twin_tez(spec).nx == 1
