"""Validation case of Sec. 3: a periodic array of n = 2 cylinders (L = 1 m,
D = 0.3 m, h = 0.01 m, dt = 23.57 ps) under a normally incident plane wave.

1. Parity: the CUDA path against the FP64 oracle at L/lambda = 0.75, 0.82,
   0.855 and 0.90 in both polarisations (stored oracle runs of 60 000 steps,
   tests/golden/make_oracle_goldens.py e2): R and T within 2e-3.
2. The S (TMz) spectrum of this discrete system: a single resonance where T
   falls to nearly zero, at L/lambda = 0.855. The position is a property of
   the discretised cylinder, not of the step count or the cell size: the
   oracle gives T = 5.5e-4 there, and halving h (200 x 1794 cells, 120 000
   steps) leaves the minimum within the 0.005 sweep step. The test bounds
   the minimum's position by that sweep step at both cell sizes. The
   paper quotes the drop "near 0.82" from a figure whose reference curve is
   not available; the difference (0.035 in L/lambda) is not explained by
   the polarisation, the cell size or the stair-cased outline and is
   recorded as a disagreement, not tested as agreement.
3. P (TEz): no drop below T = 0.9 for L/lambda < 0.9 (the field crosses the
   cylinder walls and the array barely scatters).
R + T = 1 for the lossless array in every run below the first diffraction
order (L/lambda < 0.98).
"""
import glob
import json
import os

import numpy as np
import pytest

from fdtd_inputs import config_e2
from gpu_common import lib, need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
RT_TOL = 2e-3
SWEEP_STEP = 0.005


def _goldens():
    out = []
    for js in sorted(glob.glob(os.path.join(HERE, "golden", "oracle_e2_*.json"))):
        with open(js) as f:
            out.append(json.load(f))
    return out


E2 = _goldens()


@pytest.fixture(scope="module")
def fd():
    need_gpu()
    return lib()


@pytest.mark.skipif(not E2, reason="no validation-case oracle goldens written")
def test_cylinder_array_matches_oracle(fd):
    from paper_2512_17132_gb300.campaign import run_sweep
    specs = [config_e2(g["l_over_lambda"], steps=g["steps"]).with_(
        polarization=1 if g["polarization"].startswith("P") else 0) for g in E2]
    R, T = run_sweep(specs)
    for g, r, t in zip(E2, R, T):
        print(f"{g['case']}: R {r:.6f} vs {g['R']:.6f}, T {t:.6f} vs {g['T']:.6f}")
        assert abs(r - g["R"]) <= RT_TOL and abs(t - g["T"]) <= RT_TOL


@pytest.mark.parametrize("h", [0.01, 0.005])
def test_s_resonance_position_is_mesh_converged(fd, h):
    from paper_2512_17132_gb300.campaign import run_sweep
    x = np.round(np.arange(0.70, 0.9501, SWEEP_STEP), 4)
    steps = int(round(60000 * 0.01 / h))
    R, T = run_sweep([config_e2(v, steps=steps, h=h) for v in x])
    k = int(np.argmin(T))
    print(f"h={h}: minimum T={T[k]:.2e} at L/lambda={x[k]}; T(0.75)={T[10]:.3f}")
    assert abs(x[k] - 0.855) <= SWEEP_STEP + 1e-9 and T[k] < 1e-2
    assert np.all(np.diff(T[:k + 1]) < 0) and np.all(np.diff(T[k:]) > 0)    # a single dip
    assert np.all(np.abs(R + T - 1.0) < 2e-3)                               # lossless array


def test_p_polarisation_barely_scatters(fd):
    from paper_2512_17132_gb300.campaign import run_sweep
    x = np.round(np.arange(0.50, 0.9001, 0.02), 4)
    R, T = run_sweep([config_e2(v, steps=60000).with_(polarization=1) for v in x])
    print("P:", [round(float(t), 4) for t in T])
    assert np.all(T > 0.9) and np.all(np.abs(R + T - 1.0) < 2e-3)
