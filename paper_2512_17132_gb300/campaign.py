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
    nx % 4 != 0 run one after another with the per-half-step kernels."""
    specs = list(specs)
    R = np.full(len(specs), np.nan)
    T = np.full(len(specs), np.nan)
    idx = [i for i, s in enumerate(specs) if s.nx % 4 == 0]
    rest = [i for i, s in enumerate(specs) if s.nx % 4 != 0]
    for lo in range(0, len(idx), chunk):
        part = idx[lo:lo + chunk]
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
