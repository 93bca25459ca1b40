"""The oracle's C time loops (oracle/tmz_loop.c, oracle/tez_loop.c) against
the numpy loops and the independent pins.

Each C loop repeats its numpy oracle's arithmetic cell by cell, so the two
must agree bit for bit on every field, CPML carry and DFT accumulator. The
exact discrete-lattice R/T of the config-1 slab (a frequency-domain march
that runs no time loop) and the CPML reflection bound pin each C loop on
its own as well."""
import math

import numpy as np
import pytest

from fdtd_inputs import config_c1, config_c1b
from fdtd_inputs.configs import SOURCE_NONE
from fdtd_inputs.geometry import stack_labels
from oracle import C0, TMzOracle
from oracle.fdtd_tmz import empty_twin
from oracle.fdtd_tez import TEzOracle
from oracle.fdtd_tez_c import TEzOracleC, run_rt_tez_c
from oracle.fdtd_tmz_c import TMzOracleC, run_rt_c
import pins

LAM = 550e-9
W0 = 2 * math.pi * C0 / LAM


def _same_state(a, b):
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    for k in a.dft:
        assert np.array_equal(a.dft[k], b.dft[k]), k
    for la, lb in zip(a.pml_e + a.pml_h, b.pml_e + b.pml_h):
        assert np.array_equal(la[4], lb[4])
    assert a.n == b.n


@pytest.mark.parametrize("nx,steps,threads", [(256, 350, 4), (37, 300, 1), (1, 500, 3),
                                              (64, 257, 2)])
def test_c_loop_is_bitwise_the_numpy_loop(nx, steps, threads):
    spec = config_c1b(nx=nx, steps=steps) if nx > 1 else config_c1(nx=1, steps=steps)
    a = TMzOracle(spec).run(steps)
    b = TMzOracleC(spec)
    b.run(steps // 3, threads)
    b.run(steps - steps // 3, threads)       # two calls: the state carries over
    _same_state(a, b)


def test_c_loop_from_a_random_state_without_source():
    spec = config_c1b(nx=48, steps=200).with_(source_kind=SOURCE_NONE)
    rng = np.random.default_rng(5)
    init = [rng.standard_normal((spec.ny, spec.nx)) for _ in range(3)]
    init[1] /= 376.73
    init[2] /= 376.73
    a, b = TMzOracle(spec), TMzOracleC(spec)
    a.set_fields(*init)
    b.set_fields(*init)
    a.run(200)
    b.run(200, 2)
    _same_state(a, b)


def test_c_loop_slab_rt_matches_discrete_lattice():
    base = config_c1(nx=4, steps=8000)
    spec = base.with_(labels=stack_labels(4, 256, [(40, 90, 1), (90, 215, 2)]))
    r = run_rt_c(spec, threads=2)
    idx = pins.rows_to_index(256, [(40, 90, 1.45), (90, 215, 1.42 + 1e-3j)])
    R, T = pins.lattice_stack_rt(W0, spec.dx, spec.dt, idx)
    assert abs(r["R"] - R) < 1e-5 and abs(r["T"] - T) < 1e-5


def test_c_loop_cpml_reflection():
    spec = config_c1(nx=2, steps=8000).with_(labels=np.zeros((256, 2), np.uint8))
    sim = TMzOracleC(spec).run(8000, 2)
    p_up, p_down = sim.fluxes()
    assert p_down > 0 and p_up / p_down < 1e-9


def test_c_loop_rejects_bad_rows():
    spec = config_c1b(nx=8, steps=10)
    sim = TMzOracleC(spec)
    sim.jr = spec.ny - 1                      # the Hx average would read row ny
    with pytest.raises(ValueError):
        sim.run(1)


def _same_state_tez(a, b):
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    for k in a.dft:
        assert np.array_equal(a.dft[k], b.dft[k]), k
    for la, lb in zip(a.pml_c + a.pml_x, b.pml_c + b.pml_x):
        assert np.array_equal(la[4], lb[4])
    assert a.n == b.n


@pytest.mark.parametrize("nx,steps,threads", [(256, 350, 4), (37, 300, 1), (1, 500, 3),
                                              (64, 257, 2)])
def test_tez_c_loop_is_bitwise_the_numpy_loop(nx, steps, threads):
    spec = config_c1b(nx=nx, steps=steps) if nx > 1 else config_c1(nx=1, steps=steps)
    a = TEzOracle(spec).run(steps)
    b = TEzOracleC(spec)
    b.run(steps // 3, threads)
    b.run(steps - steps // 3, threads)       # two calls: the state carries over
    _same_state_tez(a, b)


def test_tez_c_loop_per_cell_materials():
    spec = config_c1b(nx=40, steps=240)
    rng = np.random.default_rng(11)
    eps = 1.0 + 1.5 * rng.random((spec.ny, spec.nx))
    sig = 1e4 * rng.random((spec.ny, spec.nx))
    for m in (eps, sig):
        m[:spec.pml_cells + 4] = m[:spec.pml_cells + 4] * 0.0 + (1.0 if m is eps else 0.0)
    a = TEzOracle(spec, eps_r=eps, sigma=sig).run(240)
    b = TEzOracleC(spec, eps_r=eps, sigma=sig).run(240, 2)
    _same_state_tez(a, b)


def test_tez_c_loop_slab_rt_matches_discrete_lattice():
    base = config_c1(nx=4, steps=8000)
    spec = base.with_(labels=stack_labels(4, 256, [(40, 90, 1), (90, 215, 2)]))
    r = run_rt_tez_c(spec, threads=2)
    idx = pins.rows_to_index(256, [(40, 90, 1.45), (90, 215, 1.42 + 1e-3j)])
    R, T = pins.lattice_stack_rt_tez(W0, spec.dx, spec.dt, idx)
    assert abs(r["R"] - R) < 1e-5 and abs(r["T"] - T) < 1e-5


def test_tez_c_loop_cpml_reflection():
    spec = config_c1(nx=2, steps=8000).with_(labels=np.zeros((256, 2), np.uint8))
    sim = TEzOracleC(spec).run(8000, 2)
    p_up, p_down = sim.fluxes()
    assert p_down > 0 and p_up / p_down < 1e-9


def test_tez_c_loop_rejects_bad_rows():
    spec = config_c1b(nx=8, steps=10)
    sim = TEzOracleC(spec)
    sim.jt = spec.ny - 1                      # the Ex average would read row ny
    with pytest.raises(ValueError):
        sim.run(1)
