"""Pins of the Bloch-order decomposition and of the CW steady-state window
(Sec. 2.6). Right-hand sides: the Poynting fluxes of the same run (an
independent quadratic form of the monitor lines), Parseval's identity, the
exact frequency-domain lattice solution of a stack, the continuum grating
equation and obliquity k_y/k0, and the x-mirror symmetry."""
import math

import numpy as np
import pytest

from fdtd_inputs import POL_P, config_c1
from fdtd_inputs.geometry import stack_labels
from oracle import C0, TMzOracle
from oracle.bloch import bloch_orders, lattice_ky, propagating_orders
from oracle.fdtd_tez import TEzOracle, empty_twin_tez
from oracle.fdtd_tmz import empty_twin
import pins

LAM = 550e-9
W0 = 2 * math.pi * C0 / LAM


def _run(spec, steps):
    if getattr(spec, "polarization", 0):
        return TEzOracle(spec).run(steps), empty_twin_tez(spec).run(steps)
    return TMzOracle(spec).run(steps), empty_twin(spec).run(steps)


def _grating(nx=48, pol=0, centred=True, steps=5000):
    """Lossy n = 1.5 discs (kappa = 0.02, 400 nm) in air with period
    nx * 20 nm; 960 nm at nx = 48 lets orders -1, 0, 1 propagate at 550 nm."""
    ny = 256
    jj, ii = np.mgrid[0:ny, 0:nx]
    xc = nx / 2.0 if centred else nx / 3.0
    lab = (((ii + 0.5 - xc) ** 2 + (jj + 0.5 - 130.0) ** 2) <= 10.0 ** 2).astype(np.uint8)
    if not centred:
        lab[(((ii + 0.5 - 0.8 * nx) ** 2 + (jj + 0.5 - 110.0) ** 2) <= 6.0 ** 2)] = 1
    spec = config_c1(nx=nx, steps=steps).with_(
        labels=lab, materials=np.array([[1.0, 0.0], [1.5, 0.02]]), polarization=pol)
    return spec


def test_lattice_ky_tends_to_grating_equation():
    # k_y/k0 -> sqrt(1 - (m lambda / L)^2) and the propagating set -> |m| < L/lambda
    L = 2.0e-6
    for d in (20e-9, 5e-9, 1.25e-9):
        nx = int(round(L / d))
        dt = 0.5 * d / C0
        M = propagating_orders(nx, d, dt, W0)
        assert M == int(L / LAM)                         # 3 orders each side
        ky = lattice_ky(np.arange(M + 1), nx, d, dt, W0) / d
        exact = 2 * math.pi / LAM * np.sqrt(1 - (np.arange(M + 1) * LAM / L) ** 2)
        err = np.abs(ky / exact - 1).max()
        assert err < 4.0 * (2 * math.pi * d / LAM) ** 2     # O(dx^2) lattice dispersion
    assert err < 1e-4


@pytest.mark.parametrize("pol", [0, POL_P])
def test_x_uniform_stack_has_only_order_zero(pol):
    nx = 8
    spec = config_c1(nx=nx, steps=8000).with_(
        labels=stack_labels(nx, 256, [(40, 90, 1), (90, 215, 2)]), polarization=pol)
    b = bloch_orders(*_run(spec, 8000), m_max=3)
    z = b["m"] == 0
    assert np.all(b["R_paper"][~z] <= 1e-24) and np.all(b["T_paper"][~z] <= 1e-24)
    # normal incidence: |E_0|^2 / |E_inc|^2 is the power ratio (w_0 = 1), up to
    # the cross term of the CPML's ~3e-5 back-reflection at the R line
    assert b["w"][z][0] == 1.0
    assert abs(b["R_paper"][z][0] - b["R"]) < 1e-6 and abs(b["T_paper"][z][0] - b["T"]) < 1e-6
    idx = pins.rows_to_index(256, [(40, 90, 1.45), (90, 215, 1.42 + 1e-3j)])
    rt = pins.lattice_stack_rt_tez if pol else pins.lattice_stack_rt
    R, T = rt(W0, spec.dx, spec.dt, idx)
    assert abs(b["R_corr"].sum() - R) < 1e-5 and abs(b["T_corr"].sum() - T) < 1e-5


@pytest.fixture(scope="module", params=[0, POL_P])
def grating(request):
    spec = _grating(pol=request.param, centred=False)
    leaf, twin = _run(spec, spec.steps)
    return spec, bloch_orders(leaf, twin), bloch_orders(leaf, twin, m_max=spec.nx // 2 - 1)


def test_order_fluxes_sum_to_the_poynting_flux(grating):
    # Parseval: the order shares of the flux sum to the run's flux; every
    # order beyond |m| = 1 (including the Nyquist order, left out of the
    # symmetric range) is evanescent and carries no time-averaged flux in air
    spec, b, full = grating
    assert list(b["m"]) == [-1, 0, 1]
    ev = np.abs(full["m"]) > 1
    assert np.abs(full["R_flux"][ev]).sum() < 1e-6 and np.abs(full["T_flux"][ev]).sum() < 1e-6
    assert abs(full["R_flux"].sum() - b["R"]) < 1e-6 and abs(full["T_flux"].sum() - b["T"]) < 1e-6
    assert abs(b["R_flux"].sum() - b["R"]) < 1e-6 and abs(b["T_flux"].sum() - b["T"]) < 1e-6


def test_obliquity_corrected_orders_carry_the_flux(grating):
    # each propagating order is a one-way lattice plane wave at the monitors,
    # so w |E_m|^2 / |E_inc|^2 is its share of the Poynting flux
    spec, b, _ = grating
    assert np.abs(b["R_corr"] - b["R_flux"]).max() < 2e-6
    assert np.abs(b["T_corr"] - b["T_flux"]).max() < 2e-6
    assert b["R_flux"][0] > 1e-3 and b["T_flux"][0] > 1e-3      # oblique orders carry power
    # the paper's sum without the factor misses by the obliquity of orders +-1
    k = (b["w"][0] - 1.0)
    assert abs(b["T_paper"].sum() - b["T"]) > 0.5 * abs(k) * b["T_flux"][0]
    # continuum obliquity of order 1 at L = 960 nm: cos(theta) = 0.820
    ct = math.sqrt(1 - (LAM / (spec.nx * spec.dx)) ** 2)
    expect = ct if spec.polarization == 0 else 1.0 / ct
    assert abs(b["w"][0] - expect) < 5e-3


@pytest.mark.parametrize("pol", [0, POL_P])
def test_mirror_symmetric_grating_has_symmetric_orders(pol):
    spec = _grating(pol=pol, centred=True, steps=2500)
    b = bloch_orders(*_run(spec, 2500))
    for key in ("R_paper", "T_paper", "R_flux", "T_flux"):
        assert abs(b[key][0] - b[key][2]) <= 1e-12 * max(abs(b[key][0]), 1e-30) + 1e-300


@pytest.mark.parametrize("pol", [0, POL_P])
def test_cw_window_gives_the_exact_lattice_steady_state(pol):
    # raised-cosine-ramped CW source (10 periods), settle, then a DFT window
    # of an integer number of periods (55 steps each at S = 0.5, 20 nm,
    # 550 nm): the steady-state R, T of the stack on the lattice
    spec = config_c1(nx=1, steps=1).with_(
        labels=stack_labels(1, 256, [(40, 90, 1), (90, 215, 2)]), source_kind=1,
        polarization=pol)
    assert abs(LAM / (C0 * spec.dt) - 55.0) < 1e-9
    sims = [TEzOracle(spec) if pol else TMzOracle(spec),
            empty_twin_tez(spec) if pol else empty_twin(spec)]
    for s in sims:
        s.run(550 + 4400)
        s.reset_dft()
        s.run(55 * 40)
    (p_up, p_down), (_, p0) = sims[0].fluxes(), sims[1].fluxes()
    R, T = p_up / p0, p_down / p0
    idx = pins.rows_to_index(256, [(40, 90, 1.45), (90, 215, 1.42 + 1e-3j)])
    Rl, Tl = (pins.lattice_stack_rt_tez if pol else pins.lattice_stack_rt)(
        W0, spec.dx, spec.dt, idx)
    assert abs(R - Rl) < 2e-5 and abs(T - Tl) < 2e-5
