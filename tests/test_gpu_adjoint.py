"""GPU discrete adjoint (fdtd_forward_checkpointed + fdtd_backward) against
the FP64 oracle adjoint. Tolerance: 1e-3 relative (max abs error over the
map / max |reference|), per-label gradients 1e-3 relative."""
import numpy as np
import pytest

from fdtd_inputs import config_c1b, config_c5
from gpu_common import lib, need_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-3


@pytest.fixture(scope="module")
def fd():
    need_gpu()
    return lib()


def _small():
    from test_oracle_adjoint import small_spec
    return small_spec(5, nx=8, ny=40)


def _crop_c5():
    """128 x 512 crop of the config-5 stack (cuticle + lossy slab) with the
    cylinders and 1 % label noise of config 1b in its first 256 rows."""
    base = config_c5(nx=128, ny=512, steps=2500)
    lab = np.zeros((512, 128), np.uint8)
    lab[:256] = config_c1b().labels[:, :128]
    mats = np.array([[1.0, 0.0], [1.45, 0.0], [1.42, 1e-3], [2.0, 0.0]])
    return base.with_(labels=lab, materials=mats)


def _close(g, r, tol=TOL):
    return np.abs(np.asarray(g) - np.asarray(r)).max() <= tol * np.abs(np.asarray(r)).max()


@pytest.mark.parametrize("wR,wT,every", [(1.0, 0.0, 50), (0.0, 1.0, 37), (0.6, -0.4, 160)])
def test_adjoint_small_grid_matches_oracle(fd, wR, wT, every):
    from oracle.adjoint import objective_and_gradient
    spec = _small()
    steps = 160
    ref = objective_and_gradient(spec, steps, wR, wT)
    with fd.Simulation(spec) as s:
        got = s.gradient(steps, wR, wT, every)
    assert abs(got["J"] - ref["J"]) < 1e-4
    assert _close(got["g_eps"], ref["g_eps"]) and _close(got["g_sigma"], ref["g_sigma"])
    for key in ("g_n", "g_k"):
        r = ref[key][1:]
        assert np.abs(got[key][1:] - r).max() <= TOL * np.abs(r).max(), key


def test_adjoint_128x512_crop_matches_oracle(fd):
    from oracle.adjoint import objective_and_gradient
    spec = _crop_c5()
    steps = 2500
    for wR, wT in ((1.0, 0.0), (0.0, 1.0)):
        ref = objective_and_gradient(spec, steps, wR, wT)
        with fd.Simulation(spec) as s:
            got = s.gradient(steps, wR, wT, 500)
        print(f"crop wR={wR} wT={wT}: J {got['J']:.6f} / {ref['J']:.6f}, "
              f"g_eps err {np.abs(got['g_eps'] - ref['g_eps']).max() / np.abs(ref['g_eps']).max():.2e}")
        assert abs(got["J"] - ref["J"]) < 2e-3
        assert _close(got["g_eps"], ref["g_eps"]) and _close(got["g_sigma"], ref["g_sigma"])
        for key in ("g_n", "g_k"):
            r = ref[key][1:]
            assert np.abs(got[key][1:] - r).max() <= TOL * np.abs(r).max(), key


def test_map_handle_matches_label_handle(fd):
    from oracle.adjoint import maps_from_labels, objective_and_gradient
    spec = _small()
    eps, sig = maps_from_labels(spec)
    rng = np.random.default_rng(9)
    # perturb the tissue cells off the label values (a genuine per-cell map)
    eps = eps.copy()
    eps[10:30] *= 1.0 + 0.05 * rng.random((20, spec.nx))
    ref = objective_and_gradient(spec, 160, 1.0, 0.5, eps_r=eps, sigma=sig)
    with fd.Simulation(spec, eps_r=eps, sigma=sig) as s:
        got = s.gradient(160, 1.0, 0.5, 40)
    assert abs(got["J"] - ref["J"]) < 1e-4
    assert _close(got["g_eps"], ref["g_eps"]) and _close(got["g_sigma"], ref["g_sigma"])


def test_checkpoint_interval_does_not_change_the_gradient(fd):
    spec = _small()
    with fd.Simulation(spec) as s:
        a = s.gradient(160, 1.0, 0.0, 160)
        b = s.gradient(160, 1.0, 0.0, 13)
    assert a["J"] == b["J"]
    assert _close(a["g_eps"], b["g_eps"], 1e-6) and _close(a["g_sigma"], b["g_sigma"], 1e-6)


def test_backward_needs_a_checkpointed_forward(fd):
    spec = _small()
    with fd.Simulation(spec) as s:
        s.run(100)
        with pytest.raises(fd.FDTDError) as e:
            fd.fdtd_backward(s.h, 1.0, 0.0, spec.ny, spec.nx)
        assert e.value.code == fd.FDTD_ESTATE
        fd.fdtd_forward_checkpointed(s.h, 160, 40)
        s.run(1)
        with pytest.raises(fd.FDTDError):
            fd.fdtd_backward(s.h, 1.0, 0.0, spec.ny, spec.nx)


def test_autograd_functions(fd):
    import torch
    from oracle.adjoint import maps_from_labels, objective_and_gradient
    from paper_2512_17132_gb300.autograd import (reflectance_transmittance,
                                                 reflectance_transmittance_table)
    spec = _small()
    eps, sig = maps_from_labels(spec)
    e = torch.tensor(eps, requires_grad=True)
    s = torch.tensor(sig, requires_grad=True)
    rt = reflectance_transmittance(e, s, spec, 160, 40)
    loss = 0.6 * rt[0] - 0.4 * rt[1]
    loss.backward()
    ref = objective_and_gradient(spec, 160, 0.6, -0.4, eps_r=eps, sigma=sig)
    assert _close(e.grad.numpy(), ref["g_eps"]) and _close(s.grad.numpy(), ref["g_sigma"])
    tab = torch.tensor(spec.materials, requires_grad=True)
    rt = reflectance_transmittance_table(tab, spec, 160, 40)
    (rt[0] + 2.0 * rt[1]).backward()
    ref = objective_and_gradient(spec, 160, 1.0, 2.0)
    g = tab.grad.numpy()
    assert np.abs(g[1:, 0] - ref["g_n"][1:]).max() <= TOL * np.abs(ref["g_n"][1:]).max()
    assert np.abs(g[1:, 1] - ref["g_k"][1:]).max() <= TOL * np.abs(ref["g_k"][1:]).max()


def test_label_gradients_match_finite_differences_full_config5(fd):
    """Config 5 at full size (1000 x 6000, 30 000 steps, R at 550 nm): the
    adjoint's per-label gradients against central differences of the FP32
    forward (Richardson-extrapolated from steps h and h/2, h = 2e-3 for n and
    5e-4 for kappa: R oscillates with the slab's optical thickness, so the
    plain h^2 term is not negligible). These steps keep the change of R far above the FP32
    noise of a 1.8e11-update run (a one-cell step of 1e-4 would change R by
    ~1e-9, below FP32 resolution; per-cell gradients are checked against
    the FP64 oracle adjoint on the 128 x 512 crop instead)."""
    spec = config_c5()
    with fd.Simulation(spec) as s:
        g = s.gradient(spec.steps, 1.0, 0.0, 500)
    h = 2e-3

    def R_at(l, col, dv):
        m = spec.materials.copy()
        m[l, col] += dv
        with fd.Simulation(spec.with_(materials=m)) as s:
            s.run(spec.steps)
            return s.flux()[0]

    def fd_at(l, col, hh):
        if spec.materials[l, col] >= 2 * hh:                 # central difference
            return (R_at(l, col, hh) - R_at(l, col, -hh)) / (2 * hh)
        # kappa = 0: one-sided second-order difference
        return (-3 * R_at(l, col, 0.0) + 4 * R_at(l, col, hh) - R_at(l, col, 2 * hh)) / (2 * hh)

    for l in (1, 2):
        for col, key in ((0, "g_n"), (1, "g_k")):
            hh = h if col == 0 else h / 4       # kappa: smaller step, R is curved near kappa = 0
            # Richardson extrapolation of two O(h^2) estimates: error O(h^4)
            fdv = (4.0 * fd_at(l, col, hh / 2) - fd_at(l, col, hh)) / 3.0
            print(f"label {l} {key}: adjoint {g[key][l]:.6e} fd {fdv:.6e}")
            assert abs(g[key][l] - fdv) <= 1e-3 * max(abs(fdv), 1e-2), (l, key)


@pytest.mark.parametrize("spec_name", ["small", "crop", "c1b"])
def test_blocked_reverse_steps_equal_per_step_kernels(fd, spec_name):
    # K reverse steps per launch (FDTD_OPT_ADJ_BLOCK = 1..4) against one launch
    # pair per step (0): the same expressions in the same order per cell, so
    # the gradients agree bit for bit, for step counts that leave partial
    # launches at the segment ends
    if spec_name == "small":
        spec, steps, every = _small(), 160, 37
    elif spec_name == "crop":
        spec, steps, every = _crop_c5(), 1500, 250
    else:
        spec, steps, every = config_c1b(steps=1600), 1600, 173
    out = {}
    for kb in (0, 1, 2, 3, 4):
        with fd.Simulation(spec) as s:
            fd.fdtd_set_option(s.h, fd.FDTD_OPT_ADJ_BLOCK, kb)
            out[kb] = s.gradient(steps, 0.7, 0.3, every)
    for kb in (1, 2, 3, 4):
        for key in ("g_eps", "g_sigma"):
            assert np.array_equal(out[kb][key], out[0][key]), (kb, key)
        # the per-label sums are reduced with atomic FP64 adds (order not fixed)
        for key in ("g_n", "g_k"):
            np.testing.assert_allclose(out[kb][key], out[0][key], rtol=1e-12, atol=0)


def test_pair_recompute_equals_scalar_recompute(fd):
    # with <= 16 labels the forward runs code shape 5 and the adjoint's
    # recompute shape 6 (label-pair table, paired FP32); padding the material
    # table past 16 labels (the extra labels unused) forces shapes 2 and 4.
    # Both round identically, so the gradients agree bit for bit.
    spec = _crop_c5().with_(steps=1500)
    pad = np.vstack([spec.materials, np.tile([[1.3, 0.0]], (14, 1))])
    out = []
    for sp in (spec, spec.with_(materials=pad)):
        with fd.Simulation(sp) as s:
            g = s.gradient(1500, 1.0, 0.5, 250)
            out.append((g, s.stats()["variant"]))
    (ga, va), (gb, vb) = out
    assert va == 5 and vb == 2
    for key in ("g_eps", "g_sigma"):
        assert np.array_equal(ga[key], gb[key]), key
    np.testing.assert_allclose(gb["g_n"][:len(spec.materials)], ga["g_n"], rtol=1e-12, atol=0)


def _c5fd():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_c5fd.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


C5FD = _c5fd()


@pytest.mark.skipif(C5FD is None, reason="no config-5 finite-difference golden written")
def test_full_size_config5_gradient_matches_fp64_finite_differences(fd):
    # config 5 at full size (1000 x 6000, the config-1 stack), R(550 nm) over
    # the stored step count: the FP32 adjoint against FP64 central
    # differences (h = 1e-4) of the oracle at 32 random cells of the stack
    # and for n, kappa of every label. Bound: 1e-3 relative, the vector norm
    # for the cells plus a per-cell check with a floor of 1e-3 of the largest
    # entry (cells with a near-zero derivative), per label 1e-3 of the
    # largest label derivative.
    g = C5FD
    spec = config_c5(steps=g["steps"])
    assert (spec.nx, spec.ny) == (g["nx"], g["ny"])
    with fd.Simulation(spec) as s:
        got = s.gradient(g["steps"], 1.0, 0.0, 500)
    assert abs(got["R"] - g["R"]) < 1e-5
    cells = np.asarray(g["cells"])
    ge = got["g_eps"][cells[:, 0], cells[:, 1]]
    ref = np.asarray(g["g_eps"])
    rel = np.linalg.norm(ge - ref) / np.linalg.norm(ref)
    worst = np.abs(ge - ref).max() / np.abs(ref).max()
    print(f"32 cells: relative L2 {rel:.2e}, worst entry {worst:.2e} of the largest; "
          f"labels n {np.asarray(got['g_n'])} vs {np.asarray(g['g_n'])}, "
          f"kappa {np.asarray(got['g_k'])} vs {np.asarray(g['g_k'])}")
    assert rel <= TOL and worst <= TOL
    for key in ("g_n", "g_k"):
        r = np.asarray(g[key])
        assert np.abs(np.asarray(got[key]) - r).max() <= TOL * np.abs(r).max(), key
