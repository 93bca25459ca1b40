"""Helpers shared by the GPU tests: build/load the library, run the oracle
on the same seeded inputs, and compare."""
import math

import numpy as np
import pytest

ETA0 = 4.0e-7 * math.pi * 299_792_458.0


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


def need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")


def lib():
    from paper_2512_17132_gb300 import build as b
    b.build()
    from paper_2512_17132_gb300 import fdtd
    fdtd.load_library()
    return fdtd


def rel_l2(a, b, denom=None):
    d = np.linalg.norm((np.asarray(a, np.float64) - np.asarray(b, np.float64)).ravel())
    n = np.linalg.norm(np.asarray(b, np.float64).ravel()) if denom is None else denom
    return d / max(n, 1e-300)


class OracleTrace:
    """Oracle run with field snapshots at given steps and the running maximum
    of each field norm (for the relative-L2 denominator)."""

    def __init__(self, spec, snaps):
        from oracle import TMzOracle
        self.sim = TMzOracle(spec)
        self.snaps = {}
        self.max_norm = [0.0, 0.0, 0.0]
        for n in range(1, max(snaps) + 1):
            self.sim.step()
            for q, f in enumerate((self.sim.ez, self.sim.hx, self.sim.hy)):
                self.max_norm[q] = max(self.max_norm[q], float(np.linalg.norm(f)))
            if n in snaps:
                self.snaps[n] = self.sim.fields()


def field_errors(gpu_fields, ref_fields, max_norms):
    """Relative L2 error per field with the denominator
    max(||ref||, 1e-2 * max over the run of ||ref||)."""
    errs = []
    for g, r, m in zip(gpu_fields, ref_fields, max_norms):
        denom = max(np.linalg.norm(r), 1e-2 * m)
        errs.append(rel_l2(g, r, denom))
    return errs
