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
    of the E and H norms (for the relative-L2 denominator)."""

    def __init__(self, spec, snaps):
        from oracle import TMzOracle
        from oracle.fdtd_tez import TEzOracle
        pol = int(getattr(spec, "polarization", 0))
        self.sim = TEzOracle(spec) if pol else TMzOracle(spec)
        self.snaps = {}
        self.max_norm = [0.0, 0.0]
        for n in range(1, max(snaps) + 1):
            self.sim.step()
            # centre field and the edge-field vector: (Ez; Hx, Hy) or (Hz; Ex, Ey)
            c, x, y = self.sim.fields()
            e = float(np.linalg.norm(c))
            h = math.hypot(np.linalg.norm(x), np.linalg.norm(y))
            self.max_norm = [max(self.max_norm[0], e), max(self.max_norm[1], h)]
            if n in snaps:
                self.snaps[n] = (c, x, y)


def field_errors(gpu_fields, ref_fields, max_norms):
    """Relative L2 errors of the electric field Ez and of the magnetic field
    vector (Hx, Hy), each with the denominator
    max(||ref||, 1e-2 * max over the run of ||ref||). H is measured as a
    vector: in nearly x-uniform regions Hy alone is a small difference of
    nearly equal Ez values and its own ratio is ill-conditioned."""
    g = [np.asarray(x, np.float64) for x in gpu_fields]
    r = [np.asarray(x, np.float64) for x in ref_fields]
    de = np.linalg.norm(g[0] - r[0])
    ne = np.linalg.norm(r[0])
    dh = math.hypot(np.linalg.norm(g[1] - r[1]), np.linalg.norm(g[2] - r[2]))
    nh = math.hypot(np.linalg.norm(r[1]), np.linalg.norm(r[2]))
    return [de / max(ne, 1e-2 * max_norms[0], 1e-300),
            dh / max(nh, 1e-2 * max_norms[1], 1e-300)]


def component_errors(gpu_fields, ref_fields, max_norms):
    """Relative L2 error of each component on its own (Ez, Hx, Hy), with the
    same denominator rule per component family as field_errors. Reported
    beside the vector measure so that an error confined to Hy stays visible;
    Hy alone can be ill-conditioned in nearly x-uniform regions, so the
    tests print it rather than bound it."""
    g = [np.asarray(x, np.float64) for x in gpu_fields]
    r = [np.asarray(x, np.float64) for x in ref_fields]
    out = []
    for q in range(3):
        m = max_norms[0] if q == 0 else max_norms[1]
        out.append(float(np.linalg.norm(g[q] - r[q]) / max(np.linalg.norm(r[q]), 1e-2 * m, 1e-300)))
    return out
