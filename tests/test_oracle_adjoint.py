"""Pins of the oracle's discrete adjoint: the reverse step is the exact
transpose of the forward step (dot-product test), and the gradients match
brute-force central differences of the forward objective on every cell."""
import math

import numpy as np
import pytest

from fdtd_inputs import config_c1
from oracle import TMzOracle
from oracle.adjoint import (incident_power, maps_from_labels, new_adjoint_state,
                            objective, objective_and_gradient, reverse_step)


def small_spec(seed=0, nx=4, ny=36):
    """nx x ny cells at 50 nm with 4-cell CPML, a short broadband pulse and
    random lossy/lossless labels in rows 10..ny-11."""
    base = config_c1(nx=nx, steps=160)
    rng = np.random.default_rng(seed)
    lab = np.zeros((ny, nx), np.uint8)
    lab[10:ny - 10] = rng.integers(1, 4, (ny - 20, nx))
    mats = np.array([[1.0, 0.0], [1.45, 0.0], [1.42, 0.02], [1.6, 0.05]])
    dx = 50e-9
    return base.with_(nx=nx, ny=ny, dx=dx, dt=0.5 * dx / 299792458.0, pml_cells=4,
                      r_row=5, tfsf_row=7, t_row=ny - 7, labels=lab, materials=mats,
                      rel_bandwidth=0.5, t0_over_tau=2.5, pml_sigma_max=0.8 * 4 / (376.73 * dx))


def test_reverse_step_is_the_transpose_of_the_forward_step():
    spec = small_spec(1).with_(source_kind=2)
    rng = np.random.default_rng(3)
    sim = TMzOracle(spec)
    ny, nx = sim.ny, sim.nx
    x = {"E": rng.standard_normal((ny, nx)), "X": rng.standard_normal((ny, nx)),
         "Y": rng.standard_normal((ny, nx))}
    sim.ez, sim.hx, sim.hy = x["E"].copy(), x["X"].copy(), x["Y"].copy()
    x["pe"] = []
    for blk in sim.pml_e:
        blk[4][:] = rng.standard_normal(blk[4].shape)
        x["pe"].append(blk[4].copy())
    x["ph"] = []
    for blk in sim.pml_h:
        blk[4][:] = rng.standard_normal(blk[4].shape)
        x["ph"].append(blk[4].copy())
    sim.step()                                               # A x
    ax = {"E": sim.ez, "X": sim.hx, "Y": sim.hy,
          "pe": [b[4] for b in sim.pml_e], "ph": [b[4] for b in sim.pml_h]}
    lam = new_adjoint_state(sim)
    lam["lE"], lam["lX"], lam["lY"] = (rng.standard_normal((ny, nx)) for _ in range(3))
    lam["mE"] = [rng.standard_normal(m.shape) for m in lam["mE"]]
    lam["mH"] = [rng.standard_normal(m.shape) for m in lam["mH"]]
    lhs = (np.sum(lam["lE"] * ax["E"]) + np.sum(lam["lX"] * ax["X"])
           + np.sum(lam["lY"] * ax["Y"])
           + sum(np.sum(a * b) for a, b in zip(lam["mE"], ax["pe"]))
           + sum(np.sum(a * b) for a, b in zip(lam["mH"], ax["ph"])))
    reverse_step(sim, lam, 0, None)                          # A^T lambda
    rhs = (np.sum(lam["lE"] * x["E"]) + np.sum(lam["lX"] * x["X"])
           + np.sum(lam["lY"] * x["Y"])
           + sum(np.sum(a * b) for a, b in zip(lam["mE"], x["pe"]))
           + sum(np.sum(a * b) for a, b in zip(lam["mH"], x["ph"])))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


@pytest.mark.parametrize("wR,wT", [(1.0, 0.0), (0.0, 1.0)])
def test_adjoint_matches_central_differences_on_every_cell(wR, wT):
    spec = small_spec(2)
    steps = 160
    eps, sig = maps_from_labels(spec)
    g = objective_and_gradient(spec, steps, wR, wT, eps_r=eps, sigma=sig)
    pin = incident_power(spec, steps)
    # sigma steps on the scale of a unit change of n*kappa (2 w eps0 = 6e4 S/m)
    s_scale = 2.0 * (2 * math.pi * 299792458.0 / spec.lambda0) * 8.8541878128e-12
    fd_e = np.zeros_like(eps)
    fd_s = np.zeros_like(sig)
    for j in range(spec.ny):
        for i in range(spec.nx):
            h = 1e-6 * eps[j, i]
            ep, em = eps.copy(), eps.copy()
            ep[j, i] += h
            em[j, i] -= h
            fd_e[j, i] = (objective(spec, steps, wR, wT, ep, sig, pin)
                          - objective(spec, steps, wR, wT, em, sig, pin)) / (2 * h)
            hs = 1e-6 * s_scale
            sp, sm = sig.copy(), sig.copy()
            sp[j, i] += hs
            sm[j, i] -= hs
            fd_s[j, i] = (objective(spec, steps, wR, wT, eps, sp, pin)
                          - objective(spec, steps, wR, wT, eps, sm, pin)) / (2 * hs)
    assert np.abs(g["g_eps"]).max() > 0 and np.abs(g["g_sigma"]).max() > 0
    assert np.abs(g["g_eps"] - fd_e).max() <= 1e-6 * np.abs(fd_e).max()
    assert np.abs(g["g_sigma"] - fd_s).max() <= 1e-6 * np.abs(fd_s).max()


def test_label_gradient_matches_central_differences():
    spec = small_spec(4)
    steps = 160
    g = objective_and_gradient(spec, steps, 0.7, 0.3)
    pin = incident_power(spec, steps)
    for l in range(1, 4):
        for col, key in ((0, "g_n"), (1, "g_k")):
            h = 1e-6
            mp, mm = spec.materials.copy(), spec.materials.copy()
            mp[l, col] += h
            mm[l, col] -= h
            fd = (objective(spec.with_(materials=mp), steps, 0.7, 0.3, p_inc=pin)
                  - objective(spec.with_(materials=mm), steps, 0.7, 0.3, p_inc=pin)) / (2 * h)
            assert abs(g[key][l] - fd) <= 1e-6 * max(abs(fd), 1e-3), (l, key, g[key][l], fd)
