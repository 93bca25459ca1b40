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
