"""Spectral sweeps over many independent runs (wavelengths, slices,
polarisations), the way the paper builds its spectra (Sec. 4: one run per
wavelength and slice; slice results averaged). All runs of a sweep go
through one batch (fdtd_batch_*), tuned once, so they share the GPU.
"""
from __future__ import annotations

import numpy as np

from . import fdtd


def run_sweep(specs, steps=None, autotune=True, chunk=64):
    """R and T of every spec (numpy arrays in the order given). Specs with
    nx % 4 != 0 run one after another with the per-half-step kernels; the
    others go through batches of at most `chunk` runs of one polarisation."""
    specs = list(specs)
    R = np.full(len(specs), np.nan)
    T = np.full(len(specs), np.nan)
    rest = [i for i, s in enumerate(specs) if s.nx % 4 != 0]
    # one batch holds one polarisation: group the blocked runs by it
    groups = {}
    for i, s in enumerate(specs):
        if s.nx % 4 == 0:
            groups.setdefault(int(getattr(s, "polarization", 0)), []).append(i)
    parts = [g[lo:lo + chunk] for g in groups.values() for lo in range(0, len(g), chunk)]
    for part in parts:
        sims = [fdtd.Simulation(specs[i]) for i in part]
        try:
            n = steps if steps is not None else specs[part[0]].steps
            if any((steps is None and specs[i].steps != n) for i in part):
                raise ValueError("a batch runs one step count; pass `steps`")
            with fdtd.Batch(sims) as b:
                if autotune:
                    b.autotune(2)
                b.run(n)
                for i, s in zip(part, sims):
                    R[i], T[i] = s.flux()
        finally:
            for s in sims:
                s.close()
    for i in rest:
        with fdtd.Simulation(specs[i]) as s:
            s.run(steps if steps is not None else specs[i].steps)
            R[i], T[i] = s.flux()
    return R, T


def run_unpolarized(specs, steps=None, autotune=True, chunk=64):
    """Unpolarised R and T (Sec. 2.1): every spec runs once in S (TMz) and
    once in P (TEz) polarisation and the two results are averaged, both
    polarisations carrying the same incident power. Returns a dict of numpy
    arrays R, T (the means) and R_s, T_s, R_p, T_p."""
    specs = list(specs)
    both = [s.with_(polarization=fdtd.FDTD_POL_S) for s in specs] + \
           [s.with_(polarization=fdtd.FDTD_POL_P) for s in specs]
    R, T = run_sweep(both, steps=steps, autotune=autotune, chunk=chunk)
    n = len(specs)
    out = dict(R_s=R[:n], T_s=T[:n], R_p=R[n:], T_p=T[n:])
    out["R"] = 0.5 * (out["R_s"] + out["R_p"])
    out["T"] = 0.5 * (out["T_s"] + out["T_p"])
    return out
