"""Write the oracle's R, T, DFT lines and sampled fields for full-size runs.

Calls only oracle/ and fdtd_inputs/: every stored value comes from the FP64
oracle (its time loop in C, bit-identical to the numpy loop). The GPU tests
and bench.py compare the CUDA library with these files.

  python tests/golden/make_oracle_goldens.py c2 550 [450 662 800 1450] [--threads N]
      config 2: the 2000 x 12500 dicot cross-section (seed 0), 30 000 steps
      at each wavelength (nm), S polarisation, as the throughput line runs it.
  python tests/golden/make_oracle_goldens.py c2p 550 [1450 ...] [--threads N]
      the same runs in P polarisation (the TEz oracle, its time loop in C).
  python tests/golden/make_oracle_goldens.py c3crop [--threads N]
      config 3 (healthy monocot, 550 nm, dx = 15 nm) cropped to its first
      8192 rows (the whole leaf and both monitors) and 2048 columns, with R, T
      and the DFT lines after 4000 and after 60 000 steps.
  python tests/golden/make_oracle_goldens.py c3cropp [--threads N]
      the same crop in P polarisation (the TEz oracle, its time loop in C).
  python tests/golden/make_oracle_goldens.py c5fd [--threads N]
      config 5 (the config-1 stack at 1000 x 6000, 550 nm) over 6000 steps:
      R and its central differences (h = 1e-4) with respect to eps_r at 32
      random cells of the stack region (rows 30-259, seed 7) and to n and
      kappa of every label, all in FP64.
  python tests/golden/make_oracle_goldens.py e2 [--threads N]
      the validation cylinder array of Sec. 3 (100 x 897 cells, h = 0.01 m),
      60 000 steps, S and P polarisation, at L/lambda = 0.75, 0.82, 0.855
      and 0.90.

Each run writes oracle_<case>.json (scalars, with the command that made
them) and oracle_<case>.npz (the four DFT lines, complex128, in the order
Ez(r_row), Hx(r_row), Ez(t_row), Hx(t_row) for S and Hz(r_row), Ex(r_row),
Hz(t_row), Ex(t_row) for P, and the fields Ez, Hx, Hy (S) or Hz, Ex, Ey (P)
at 4096 cells drawn with numpy's default_rng(2024), with their flat
indices, under the keys ez, hx, hy).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from fdtd_inputs import config_c2, config_c3, config_c5, config_e2, crop_layout  # noqa: E402
from oracle import eps_sigma  # noqa: E402
from oracle.fdtd_tez import empty_twin_tez  # noqa: E402
from oracle.fdtd_tez_c import TEzOracleC  # noqa: E402
from oracle.fdtd_tmz import empty_twin  # noqa: E402
from oracle.fdtd_tmz_c import TMzOracleC  # noqa: E402

N_SAMPLES = 4096
SAMPLE_SEED = 2024


def sample_index(ny, nx):
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(ny * nx, N_SAMPLES, replace=False))


def c3_crop_spec(**kw):
    """Config 3 healthy at 550 nm, first 8192 rows and 2048 columns."""
    return crop_layout(config_c3(550e-9, **kw), 8192, 2048)


def _record(name, spec, leaf, twin, steps, wall, threads, cmd, extra=None):
    p_up, p_down = leaf.fluxes()
    p_inc = twin.fluxes()[1] * spec.nx

    def ratio(x):
        # None until the incident pulse has reached t_row (P_inc = 0)
        return x / p_inc if p_inc > 0.0 else None

    rec = dict(
        case=name, nx=spec.nx, ny=spec.ny, dx=spec.dx, dt=spec.dt, steps=int(steps),
        lambda0=spec.lambda0, r_row=spec.r_row, t_row=spec.t_row, tfsf_row=spec.tfsf_row,
        polarization="P (TEz)" if getattr(spec, "polarization", 0) else "S (TMz)",
        R=ratio(p_up), T=ratio(p_down),
        A=None if p_inc <= 0.0 else 1.0 - (p_up + p_down) / p_inc, p_up=p_up, p_down=p_down, p_inc=p_inc,
        oracle=("FP64 oracle (TEzOracle state, C time loop TEzOracleC)"
                if getattr(spec, "polarization", 0) else
                "FP64 oracle (TMzOracle state, C time loop TMzOracleC)"),
        threads=int(threads), wall_s=round(wall, 1), command=cmd)
    if extra:
        rec.update(extra)
    idx = sample_index(spec.ny, spec.nx)
    d = leaf.dft
    fields = leaf.fields()                   # (Ez, Hx, Hy) or, for P, (Hz, Ex, Ey)
    order = (("h_r", "e_r", "h_t", "e_t") if getattr(spec, "polarization", 0)
             else ("e_r", "h_r", "e_t", "h_t"))
    np.savez_compressed(
        os.path.join(HERE, f"oracle_{name}.npz"),
        dft=np.stack([d[k] for k in order]),
        idx=idx, ez=fields[0].ravel()[idx], hx=fields[1].ravel()[idx],
        hy=fields[2].ravel()[idx], max_abs=np.array([np.abs(f).max() for f in fields]))
    with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps({k: rec[k] for k in ("case", "steps", "R", "T", "A", "wall_s")}), flush=True)


def run_c2(lam_nm, threads):
    spec = config_c2(lam_nm * 1e-9)
    t = time.time()
    leaf = TMzOracleC(spec).run(spec.steps, threads)
    twin = empty_twin(spec).run(spec.steps)
    _record(f"c2_{lam_nm:g}nm", spec, leaf, twin, spec.steps, time.time() - t, threads,
            f"python tests/golden/make_oracle_goldens.py c2 {lam_nm:g} --threads {threads}",
            dict(seed=0))


def run_c2p(lam_nm, threads):
    spec = config_c2(lam_nm * 1e-9).with_(polarization=1)
    t = time.time()
    leaf = TEzOracleC(spec).run(spec.steps, threads)
    twin = empty_twin_tez(spec).run(spec.steps)
    _record(f"c2p_{lam_nm:g}nm", spec, leaf, twin, spec.steps, time.time() - t, threads,
            f"python tests/golden/make_oracle_goldens.py c2p {lam_nm:g} --threads {threads}",
            dict(seed=0))


def run_c3crop(threads, pol=0):
    spec = c3_crop_spec().with_(polarization=pol)
    name = "c3cropp" if pol else "c3crop"
    t = time.time()
    leaf = TEzOracleC(spec) if pol else TMzOracleC(spec)
    twin = empty_twin_tez(spec) if pol else empty_twin(spec)
    done = 0
    for steps in (4000, 60000):
        leaf.run(steps - done, threads)
        twin.run(steps - done)
        done = steps
        _record(f"{name}_{steps}", spec, leaf, twin, steps, time.time() - t, threads,
                f"python tests/golden/make_oracle_goldens.py {name} --threads {threads}",
                dict(seed=0, crop="config 3 healthy, rows 0-8191, columns 0-2047"))


E2_POINTS = (0.75, 0.82, 0.855, 0.90)


def run_e2(threads):
    for pol in (0, 1):
        for x in E2_POINTS:
            spec = config_e2(x, steps=60000).with_(polarization=pol)
            t = time.time()
            if pol:
                leaf = TEzOracleC(spec).run(spec.steps, threads)
                twin = empty_twin_tez(spec).run(spec.steps)
            else:
                leaf = TMzOracleC(spec).run(spec.steps, threads)
                twin = empty_twin(spec).run(spec.steps)
            _record(f"e2_{'SP'[pol]}_{x:g}", spec, leaf, twin, spec.steps, time.time() - t,
                    threads,
                    f"python tests/golden/make_oracle_goldens.py e2 --threads {threads}",
                    dict(l_over_lambda=x))


def c5fd_cells(ny, nx):
    """The 32 cells of the config-5 finite differences: rows 30-259 (the
    stack between the monitors), any column, numpy default_rng(7)."""
    rng = np.random.default_rng(7)
    return np.stack([rng.integers(30, 260, 32), rng.integers(0, nx, 32)], axis=1)


def run_c5fd(threads, steps=6000, h=1e-4, spec=None, out_name="c5fd"):
    spec = config_c5(steps=steps) if spec is None else spec
    t0 = time.time()
    twin = empty_twin(spec).run(steps)
    p_inc = twin.fluxes()[1] * spec.nx
    omega = 2.0 * np.pi * 299_792_458.0 / spec.lambda0
    mats = np.asarray(spec.materials, dtype=np.float64)

    def reflectance(eps, sig):
        leaf = TMzOracleC(spec, eps_r=eps, sigma=sig).run(steps, threads)
        return leaf.fluxes()[0] / p_inc

    def maps(m):
        return eps_sigma(m[spec.labels, 0], m[spec.labels, 1], omega)

    eps0, sig0 = maps(mats)
    R0 = reflectance(eps0, sig0)
    cells = c5fd_cells(spec.ny, spec.nx)
    g_eps = []
    for j, i in cells:
        e = eps0.copy()
        e[j, i] += h
        rp = reflectance(e, sig0)
        e[j, i] -= 2.0 * h
        rm = reflectance(e, sig0)
        g_eps.append((rp - rm) / (2.0 * h))
        print(f"cell ({j}, {i}): dR/deps = {g_eps[-1]:.9e}", flush=True)
    g_n, g_k = [], []
    for lab in range(len(mats)):
        for col, out in ((0, g_n), (1, g_k)):
            m = mats.copy()
            m[lab, col] += h
            rp = reflectance(*maps(m))
            m[lab, col] -= 2.0 * h
            rm = reflectance(*maps(m))
            out.append((rp - rm) / (2.0 * h))
    rec = dict(case=out_name, nx=spec.nx, ny=spec.ny, steps=int(steps), lambda0=spec.lambda0,
               h=h, R=R0, cells=cells.tolist(), g_eps=g_eps, g_n=g_n, g_k=g_k,
               oracle="FP64 oracle (TMzOracle state, C time loop TMzOracleC), central differences",
               threads=int(threads), wall_s=round(time.time() - t0, 1),
               command=f"python tests/golden/make_oracle_goldens.py c5fd --threads {threads}")
    with open(os.path.join(HERE, f"oracle_{out_name}.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps({k: rec[k] for k in ("case", "steps", "R", "wall_s")}), flush=True)


def main(argv):
    threads = os.cpu_count() or 1
    if "--threads" in argv:
        k = argv.index("--threads")
        threads = int(argv[k + 1])
        argv = argv[:k] + argv[k + 2:]
    case = argv[0]
    if case == "c2":
        for lam in argv[1:] or ["550"]:
            run_c2(float(lam), threads)
    elif case == "c2p":
        for lam in argv[1:] or ["550"]:
            run_c2p(float(lam), threads)
    elif case == "c3crop":
        run_c3crop(threads)
    elif case == "c3cropp":
        run_c3crop(threads, pol=1)
    elif case == "e2":
        run_e2(threads)
    elif case == "c5fd":
        run_c5fd(threads)
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv[1:])
