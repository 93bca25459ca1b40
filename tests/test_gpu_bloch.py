"""Bloch-order decomposition and CW steady-state window through the C ABI
against the FP64 oracle (Sec. 2.6). Tolerances: order quantities within
2e-5 absolute (they are ratios of O(0.1)), the lattice wavenumbers and
obliquity factors to 1e-12 (host FP64 on both sides), Parseval at full size
to 1e-6 relative."""
import math

import numpy as np
import pytest

from fdtd_inputs import POL_P, config_c1, config_c2
from fdtd_inputs.geometry import stack_labels
from gpu_common import lib, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    need_gpu()
    return lib()


def _grating(pol, steps=5000):
    nx, ny = 48, 256
    jj, ii = np.mgrid[0:ny, 0:nx]
    lab = (((ii + 0.5 - nx / 3.0) ** 2 + (jj + 0.5 - 130.0) ** 2) <= 10.0 ** 2).astype(np.uint8)
    lab[(((ii + 0.5 - 0.8 * nx) ** 2 + (jj + 0.5 - 110.0) ** 2) <= 6.0 ** 2)] = 1
    return config_c1(nx=nx, steps=steps).with_(
        labels=lab, materials=np.array([[1.0, 0.0], [1.5, 0.02]]), polarization=pol)


def _oracle(spec, steps):
    from oracle import TMzOracle
    from oracle.fdtd_tez import TEzOracle, empty_twin_tez
    from oracle.fdtd_tmz import empty_twin
    if spec.polarization:
        return TEzOracle(spec).run(steps), empty_twin_tez(spec).run(steps)
    return TMzOracle(spec).run(steps), empty_twin(spec).run(steps)


@pytest.mark.parametrize("pol", [0, POL_P])
@pytest.mark.parametrize("kernel", [1, 2])
def test_bloch_orders_match_oracle(fd, pol, kernel):
    from oracle.bloch import bloch_orders, propagating_orders
    spec = _grating(pol)
    leaf, twin = _oracle(spec, spec.steps)
    with fd.Simulation(spec, kernel=kernel) as s:
        s.run(spec.steps)
        M = fd.fdtd_bloch_propagating(s.h)
        assert M == propagating_orders(spec.nx, spec.dx, spec.dt, leaf.omega) == 1
        got = s.bloch(5)
        R, T = s.flux()
    ref = bloch_orders(leaf, twin, m_max=5)
    assert np.array_equal(got["m"], ref["m"])
    for key in ("R_flux", "T_flux", "R_paper", "T_paper", "R_corr", "T_corr"):
        assert np.abs(got[key] - ref[key]).max() < 2e-5, (key, got[key], ref[key])
    np.testing.assert_allclose(got["w"], ref["w"], rtol=1e-12, atol=0)
    prop = np.isfinite(ref["ky"])
    assert np.array_equal(np.isfinite(got["ky"]), prop)
    np.testing.assert_allclose(got["ky"][prop], ref["ky"][prop], rtol=1e-12)
    # the corrected propagating orders carry the run's flux
    assert abs(got["R_corr"][prop].sum() - R) < 1e-5 and abs(got["T_corr"][prop].sum() - T) < 1e-5


@pytest.mark.parametrize("pol", [0, POL_P])
def test_cw_window_matches_oracle_and_lattice(fd, pol):
    import pins
    from oracle import C0
    spec = config_c1(nx=4, steps=1).with_(
        labels=stack_labels(4, 256, [(40, 90, 1), (90, 215, 2)]), source_kind=1,
        polarization=pol)
    leaf, twin = _oracle(spec, 550 + 4400)
    for o in (leaf, twin):
        o.reset_dft()
        o.run(55 * 40)
    p0 = twin.fluxes()[1] * spec.nx
    Ro, To = leaf.fluxes()[0] / p0, leaf.fluxes()[1] / p0
    for kernel in (1, 2):
        with fd.Simulation(spec, kernel=kernel) as s:
            s.run(550 + 4400)
            s.reset_dft()
            s.run(55 * 40)
            R, T = s.flux()
        assert abs(R - Ro) < 1e-5 and abs(T - To) < 1e-5, (kernel, R, Ro, T, To)
    w0 = 2 * math.pi * C0 / spec.lambda0
    idx = pins.rows_to_index(256, [(40, 90, 1.45), (90, 215, 1.42 + 1e-3j)])
    Rl, Tl = (pins.lattice_stack_rt_tez if pol else pins.lattice_stack_rt)(
        w0, spec.dx, spec.dt, idx)
    assert abs(R - Rl) < 3e-5 and abs(T - Tl) < 3e-5


def test_bloch_argument_errors(fd):
    spec = _grating(0, steps=10)
    with fd.Simulation(spec) as s:
        s.run(10)
        with pytest.raises(fd.FDTDError) as e:
            fd.fdtd_bloch_orders(s.h, 24)              # 2 m + 1 > nx
        assert e.value.code == fd.FDTD_EINVAL
        with pytest.raises(fd.FDTDError):
            fd.fdtd_bloch_orders(s.h, -1)
        assert fd.fdtd_bloch_orders(s.h, 23)["m"][-1] == 23


@pytest.mark.parametrize("pol", [0, POL_P])
def test_parseval_at_full_size_config2(fd, pol):
    # the 1999 orders m = -999..999 of the 2000-column lines (all but the
    # Nyquist order, which a symmetric range cannot hold): their shares sum
    # to R and T up to that order's grid-scale share
    spec = config_c2().with_(polarization=pol)          # 30 000 steps: the pulse reaches t_row
    with fd.Simulation(spec) as s:
        s.run(spec.steps)
        R, T = s.flux()
        b = s.bloch(999)
        M = fd.fdtd_bloch_propagating(s.h)
    assert M == int(spec.nx * spec.dx / spec.lambda0)        # 72 at 550 nm
    print(f"pol {pol}: R {R:.9e} sum {b['R_flux'].sum():.9e}; T {T:.3e} sum {b['T_flux'].sum():.3e}")
    assert abs(b["R_flux"].sum() - R) <= 1e-6 * abs(R)
    assert abs(b["T_flux"].sum() - T) <= 1e-6 * max(abs(T), 1e-6)
    assert R > 1e-3 and T > 0
