"""Pins of the FP64 oracle against closed forms, invariants and the paper's
worked numbers. None of these compare the oracle with itself: each value on
the right-hand side comes from mathematics the oracle does not execute
(frequency-domain lattice recurrences, continuum transfer matrices, the
dispersion relation of a standing wave, exact symmetries)."""
import json
import math
import os

import numpy as np
import pytest

from fdtd_inputs import config_c1, config_c1b, courant_dt, C0 as C0_IN
from fdtd_inputs.geometry import stack_labels
from oracle import (C0, EPS0, MU0, eps_sigma, lossy_coefficients, cpml_profile,
                    source_waveform, IncidentLine, TMzOracle, run_rt)
from oracle.fdtd_tmz import empty_twin
import pins

HERE = os.path.dirname(os.path.abspath(__file__))
LAM = 550e-9
W0 = 2 * math.pi * C0 / LAM


def _spec_1d(ny=256, layers=(), steps=4000, **kw):
    """x-uniform single-column spec with c1's rows and CPML."""
    base = config_c1(nx=1, steps=steps)
    lab = stack_labels(1, ny, [(r0, r1, v) for r0, r1, v in layers])
    return base.with_(ny=ny, labels=lab, **kw)


# -- constants and coefficients ---------------------------------------------------------

def test_constants_agree_with_input_module():
    assert C0 == C0_IN
    assert abs(EPS0 * MU0 * C0 * C0 - 1.0) < 1e-15


def test_eps_sigma_is_the_complex_square():
    # Sec. 2.2: eps_r + i sigma/(w eps0) = (n + i kappa)^2
    rng = np.random.default_rng(0)
    n = rng.uniform(1.0, 2.0, 50)
    k = rng.uniform(0.0, 0.5, 50)
    e, s = eps_sigma(n, k, W0)
    z = (n + 1j * k) ** 2
    np.testing.assert_allclose(e, z.real, rtol=1e-14)
    np.testing.assert_allclose(s / (W0 * EPS0), z.imag, rtol=1e-14)


def test_lossy_coefficients_limits_and_order():
    # Sec. 2.3: no loss -> pure leapfrog; the loss factor is the (1,1) Pade
    # approximant of exp(-sigma dt/(eps0 eps_r)), so it matches to O(b^3).
    ce, ch = lossy_coefficients(np.array([2.0]), np.array([0.0]), 1e-17)
    assert ce[0] == 1.0 and ch[0] == 1.0
    dt = courant_dt(20e-9)
    for sig in (1e3, 1e4, 1e5):
        b = sig * dt / (2 * EPS0 * 2.0)
        ce, _ = lossy_coefficients(2.0, sig, dt)
        assert abs(ce - math.exp(-2 * b)) <= 0.2 * (2 * b) ** 3
    ce, _ = lossy_coefficients(1.0, 1e12, dt)
    assert -1.0 < ce < -0.99


def test_cpml_profile_special_cases():
    dt = courant_dt(20e-9)
    b, c, k = cpml_profile(np.array([0.0]), 16, 3, 4e5, 1.0, 1500.0, dt)
    assert c[0] == 0.0 and k[0] == 1.0          # interface: no stretching
    # alpha is alpha_max at the interface and falls to 0 at the outer wall
    assert abs(b[0] - math.exp(-1500.0 * dt / EPS0)) < 1e-15
    b, c, k = cpml_profile(np.array([16.0]), 16, 3, 4e5, 3.0, 1500.0, dt)
    assert abs(b[0] - math.exp(-4e5 / 3.0 * dt / EPS0)) < 1e-15 and k[0] == 3.0
    # kappa = 1 and alpha = 0 reduce the CFS-PML to the classical PML: c = b - 1
    d = np.linspace(0.5, 15.5, 16)
    b, c, k = cpml_profile(d, 16, 3, 4e5, 1.0, 0.0, dt)
    np.testing.assert_allclose(c, b - 1.0, rtol=1e-13)
    np.testing.assert_allclose(b, np.exp(-4e5 * (d / 16) ** 3 * dt / EPS0), rtol=1e-13)
    assert np.all(np.diff(b) < 0)


# -- source -------------------------------------------------------------------------------

def test_pulse_spectrum_fwhm_is_ten_percent():
    dt = courant_dt(20e-9)
    n = np.arange(20000)
    s = np.array([source_waveform(0, (m + 0.5) * dt, LAM, 0.1, 5.0) for m in n])
    f0 = C0 / LAM
    f = np.linspace(0.8 * f0, 1.2 * f0, 4001)
    S = np.abs(np.exp(2j * np.pi * np.outer(f, (n + 0.5) * dt)) @ s)
    half = f[S >= S.max() / 2]
    assert abs((half[-1] - half[0]) / f0 - 0.1) < 2e-3
    assert abs(f[np.argmax(S)] / f0 - 1.0) < 1e-3


def test_cw_source_ramp_is_continuous():
    f0 = C0 / LAM
    tr = 10 / f0
    a = source_waveform(1, tr * (1 - 1e-9), LAM)
    b = source_waveform(1, tr * (1 + 1e-9), LAM)
    assert abs(a - b) < 1e-6
    assert source_waveform(1, 0.0, LAM) == 0.0
    assert source_waveform(2, 1e-15, LAM) == 0.0


def test_incident_line_is_one_lattice_cell_of_propagation():
    # Semi-infinite lattice driven at cell 0: the steady-state response at
    # cell 1 is the source spectrum times exp(i k~ dx) (outgoing lattice wave).
    dx = 20e-9
    dt = courant_dt(dx)
    line = IncidentLine(dx, dt, 0, LAM, 0.1, 5.0)
    N = 5000
    e1, s = np.empty(N), np.empty(N)
    for m in range(N):
        line.advance_e()
        e1[m] = line.e_inc()
        s[m] = line.ez[0]
        line.advance_h()
    t = (np.arange(N) + 0.5) * dt
    for w in (W0, 0.95 * W0, 1.05 * W0):
        ratio = (np.exp(1j * w * t) @ e1) / (np.exp(1j * w * t) @ s)
        k = pins.lattice_wavenumber(w, dx, dt)
        assert abs(ratio - np.exp(1j * k * dx)) < 1e-9


# -- plane wave in vacuum: dispersion and TF/SF ------------------------------------------

def test_vacuum_dispersion_and_zero_sf_leakage():
    ny, steps = 2000, 3600
    spec = _spec_1d(ny=ny, steps=steps, r_row=300, t_row=310)
    sim = TMzOracle(spec)
    leak, peak = 0.0, 0.0
    for _ in range(steps):
        sim.step()
        leak = max(leak, np.abs(sim.ez[: spec.tfsf_row]).max(),
                   np.abs(sim.hx[: spec.tfsf_row + 1]).max() * 376.73)
        peak = max(peak, np.abs(sim.ez).max())
    assert leak <= 1e-12 * peak
    ratio = sim.dft["e_t"][0] / sim.dft["e_r"][0]
    k = 2.0 / spec.dx * math.asin(math.sin(W0 * spec.dt / 2) / spec.courant)
    assert abs(ratio - np.exp(1j * k * 10 * spec.dx)) < 1e-8
    # a one-way lattice wave: the row-averaged Hx phasor (time stamps n+1)
    # is -cos(k dx/2)/eta0 times the Ez phasor (time stamps n+1/2)
    for row in ("r", "t"):
        eh = sim.dft["h_" + row][0] / sim.dft["e_" + row][0] * (MU0 * C0)
        assert abs(eh + math.cos(k * spec.dx / 2)) < 1e-9
    assert abs(k / (2 * math.pi / LAM) - 1 - 1.6407e-3) < 1e-6


# -- 1D stacks: lattice R/T, energy, Beer-Lambert, Fresnel, CPML -------------------------

C1_LAYERS = [(40, 90, 1), (90, 215, 2)]


def test_slab_rt_matches_discrete_lattice():
    spec = _spec_1d(layers=C1_LAYERS, steps=8000)
    r = run_rt(spec)
    idx = pins.rows_to_index(256, [(40, 90, 1.45), (90, 215, 1.42 + 1e-3j)])
    R, T = pins.lattice_stack_rt(W0, spec.dx, spec.dt, idx)
    assert abs(r["R"] - R) < 1e-5 and abs(r["T"] - T) < 1e-5
    assert abs(R - 0.06867) < 1e-5 and abs(T - 0.87600) < 1e-5


def test_lossless_slab_conserves_energy():
    spec = _spec_1d(layers=C1_LAYERS, steps=8000)
    spec = spec.with_(materials=np.array([[1.0, 0.0], [1.45, 0.0], [1.42, 0.0]]))
    r = run_rt(spec)
    assert abs(r["R"] + r["T"] - 1.0) < 1e-5
    idx = pins.rows_to_index(256, [(40, 90, 1.45), (90, 215, 1.42)])
    R, T = pins.lattice_stack_rt(W0, spec.dx, spec.dt, idx)
    assert abs(r["R"] - R) < 1e-5


def test_beer_lambert_index_matched_layer():
    # n = 1, kappa = 1e-3 over 2.5 um: T ~ exp(-4 pi kappa d / lambda) = 0.94448
    spec = _spec_1d(layers=[(90, 215, 1)], steps=6000)
    spec = spec.with_(materials=np.array([[1.0, 0.0], [1.0, 1e-3]]))
    r = run_rt(spec)
    assert abs(r["T"] - math.exp(-4 * math.pi * 1e-3 * 2.5e-6 / LAM)) < 3e-4
    idx = pins.rows_to_index(256, [(90, 215, 1.0 + 1e-3j)])
    R, T = pins.lattice_stack_rt(W0, spec.dx, spec.dt, idx)
    assert abs(r["T"] - T) < 1e-5 and r["R"] < 1e-5


def test_fresnel_half_space():
    # air / n = 1.45 half-space (the dielectric runs through the bottom CPML):
    # the exact lattice reflection, which tends to the continuum Fresnel value
    # 0.033736 as dx -> 0 (checked in test_lattice_tends_to_continuum)
    ny = 256
    spec = _spec_1d(ny=ny, layers=[(120, ny, 1)], steps=6000)
    spec = spec.with_(materials=np.array([[1.0, 0.0], [1.45, 0.0]]))
    r = run_rt(spec)
    R_lat, _ = pins.lattice_stack_rt(W0, spec.dx, spec.dt,
                                     pins.rows_to_index(200, [(100, 200, 1.45)]))
    assert abs(r["R"] - R_lat) < 1e-5
    assert abs(r["R"] - ((1.45 - 1) / 2.45) ** 2) < 2e-3


def test_lattice_tends_to_continuum():
    # the pins themselves: lattice R/T -> Airy / Fresnel under refinement
    errs_slab, errs_if = [], []
    for d in (20e-9, 10e-9, 5e-9):
        dt = 0.5 * d / C0
        n1, n2 = int(round(1e-6 / d)), int(round(2.5e-6 / d))
        idx = pins.rows_to_index(n1 + n2 + 20, [(10, 10 + n1, 1.45),
                                                (10 + n1, 10 + n1 + n2, 1.42 + 1e-3j)])
        R, T = pins.lattice_stack_rt(W0, d, dt, idx)
        Rc, Tc = pins.continuum_stack_rt(LAM, [(1e-6, 1.45), (2.5e-6, 1.42 + 1e-3j)])
        errs_slab.append(abs(R - Rc) + abs(T - Tc))
        Ri, _ = pins.lattice_stack_rt(W0, d, dt, pins.rows_to_index(40, [(20, 40, 1.45)]))
        errs_if.append(abs(Ri - ((1.45 - 1) / 2.45) ** 2))
    assert errs_slab[0] / errs_slab[1] > 3.5 and errs_slab[1] / errs_slab[2] > 3.5
    assert errs_if[0] > errs_if[1] > errs_if[2]
    assert abs(Rc - 0.04012) < 1e-5 and abs(Tc - 0.90367) < 1e-5


@pytest.mark.parametrize("kappa_max", [1.0, 4.0])
def test_cpml_reflection_below_1e_minus_4(kappa_max):
    spec = _spec_1d(layers=[], steps=8000, pml_kappa_max=kappa_max)
    sim = empty_twin(spec).run(8000)
    p_up, p_down = sim.fluxes()
    # reflected power of the bottom CPML, normalised to the incident power:
    # far below the 1e-4 target (|r| < 3e-5 at 16 cells)
    assert p_up / p_down < 1e-9
    assert p_down > 0


# -- 2D pins: eigenmode closed form, symmetries ---------------------------------------------

def _cavity_spec(nx, ny, courant=0.5):
    base = config_c1(nx=nx, steps=1)
    return base.with_(ny=ny, nx=nx, dt=courant_dt(base.dx, courant),
                      labels=np.zeros((ny, nx), np.uint8),
                      materials=np.array([[1.0, 0.0]]), pml_cells=0,
                      source_kind=2, tfsf_row=2, r_row=1, t_row=ny - 3)


@pytest.mark.parametrize("mx,my,courant", [(3, 2, 0.5), (1, 5, 0.5), (12, 9, 0.7071)])
def test_cavity_eigenmode_closed_form(mx, my, courant):
    # Periodic x, Hx = 0 on the top and bottom walls: cos(kx x) cos(ky s)
    # standing waves oscillate at the 2D lattice frequency
    # sin^2(w dt/2) = S^2 (sin^2(kx dx/2) + sin^2(ky dx/2)).
    nx, ny = 24, 18
    spec = _cavity_spec(nx, ny, courant)
    dx, dt, S = spec.dx, spec.dt, spec.courant
    kx = 2 * math.pi * mx / (nx * dx)
    ky = math.pi * my / (ny * dx)
    s2 = S * S * (math.sin(kx * dx / 2) ** 2 + math.sin(ky * dx / 2) ** 2)
    w = 2.0 * math.asin(math.sqrt(s2)) / dt
    i = np.arange(nx)
    j = np.arange(ny)
    shape = np.outer(np.cos(ky * (j + 0.5) * dx), np.cos(kx * (i + 0.5) * dx + 0.3))
    sim = TMzOracle(spec)
    sim.set_fields(math.cos(w * dt / 2) * shape, np.zeros((ny, nx)), np.zeros((ny, nx)))
    for n in range(400):
        sim.step()
        expect = math.cos(w * (n + 0.5) * dt) * shape
        assert np.abs(sim.ez - expect).max() < 1e-11


def test_x_shift_equivariance_is_exact():
    spec = config_c1b(steps=1300)
    a = TMzOracle(spec).run(1300)
    b = TMzOracle(spec.with_(labels=np.roll(spec.labels, 37, axis=1))).run(1300)
    for fa, fb in zip(a.fields(), b.fields()):
        assert np.array_equal(np.roll(fa, 37, axis=1), fb)


def test_mirror_symmetry_is_exact():
    from fdtd_inputs.geometry import c1b_labels
    spec = config_c1b(steps=1300)
    lab = c1b_labels(256, noise=0.0)                            # cylinders only
    assert np.array_equal(lab, lab[:, ::-1])
    sim = TMzOracle(spec.with_(labels=lab)).run(1300)
    ez, hx, hy = sim.fields()
    assert np.abs(ez).max() > 0.1
    assert np.array_equal(ez, ez[:, ::-1]) and np.array_equal(hx, hx[:, ::-1])
    # Hy on edge i mirrors to edge (nx - i) mod nx with a sign change
    assert np.array_equal(hy, -np.roll(hy[:, ::-1], 1, axis=1))


def test_single_column_equals_uniform_wide_grid():
    a = TMzOracle(config_c1(nx=1, steps=600)).run(600)
    b = TMzOracle(config_c1(nx=5, steps=600)).run(600)
    for fa, fb in zip(a.fields(), b.fields()):
        assert np.array_equal(np.repeat(fa, 5, axis=1), fb)


def test_cfl_limit_is_enforced():
    spec = config_c1(nx=1, steps=1)
    with pytest.raises(ValueError):
        TMzOracle(spec.with_(dt=courant_dt(spec.dx, 0.7072)))


# -- the paper's worked numbers -------------------------------------------------------------

def test_paper_worked_numbers():
    with open(os.path.join(HERE, "golden", "paper_worked_numbers.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        if case["kind"] == "courant_dt":
            c = case.get("c", C0)
            dt = case["courant"] * case["h"] / c
            assert abs(dt - case["dt"]) <= case["tol"], case
        elif case["kind"] == "periods":
            n_per = case["steps"] * case["dt"] * case.get("c_paper", C0) / case["lambda"]
            assert abs(n_per - case["periods"]) <= case["tol"], case
        elif case["kind"] == "lambda_min":
            assert abs(case["lambda0"] / case["n"] - case["value"]) <= case["tol"]
        elif case["kind"] == "cells":
            assert abs(case["nx"] * case["ny"] - case["value"]) <= case["tol"]
