"""The TEz oracle with its time loop in plain C (oracle/tez_loop.c).

TEST INFRASTRUCTURE, like the rest of this package. TEzOracleC is the numpy
oracle (fdtd_tez.TEzOracle: same constructor, state, edge coefficients,
CPML profiles, incident line, DFT phases and fluxes); only run(steps) hands
the leapfrog loop to the C function, which repeats the numpy oracle's
arithmetic operation for operation, cell by cell, on all host cores. The
two agree bit for bit (tests/test_oracle_c.py), so every pin of the numpy
TEz oracle carries over, and full-size P-polarised grids finish in minutes
per thousand steps instead of hours.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .fdtd_tez import TEzOracle, empty_twin_tez
from .fdtd_tmz import SOURCE_NONE
from .fdtd_tmz_c import compile_loop, pml_pack, pml_unpack

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tez_loop.c")
LIB = os.path.join(HERE, "_tez_loop.so")


class _Args(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_double),
                ("ch_curl", ctypes.c_double), ("js", ctypes.c_int32), ("tfsf", ctypes.c_int32),
                ("jr", ctypes.c_int32), ("jt", ctypes.c_int32), ("threads", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the TEz C loop."""
    return compile_loop(SRC, LIB, force)


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.tez_loop_run.restype = ctypes.c_int
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _full(a, ny, nx):
    return np.ascontiguousarray(np.broadcast_to(a, (ny, nx)), dtype=np.float64)


class TEzOracleC(TEzOracle):
    """TEzOracle whose run(steps) advances with the C loop."""

    threads = os.cpu_count() or 1

    def run(self, steps, threads=None):
        steps = int(steps)
        if steps <= 0:
            return self
        # incident samples and DFT phases, taken exactly as TEzOracle.step() takes them
        e_inc = np.empty(steps)
        h_inc = np.empty(steps)
        ph_h = np.empty(2 * steps)
        ph_e = np.empty(2 * steps)
        for m in range(steps):
            n = self.n + m
            e_inc[m] = self.inc.e_inc()
            self.inc.advance_h()
            h_inc[m] = self.inc.h_inc()
            self.inc.advance_e()
            pH = np.exp(1j * self.omega * ((n + 0.5) * self.dt))
            pE = np.exp(1j * self.omega * ((n + 1.0) * self.dt))
            ph_h[2 * m], ph_h[2 * m + 1] = pH.real, pH.imag
            ph_e[2 * m], ph_e[2 * m + 1] = pE.real, pE.imag
        for name in ("hz", "ex", "ey"):
            setattr(self, name, np.ascontiguousarray(getattr(self, name), dtype=np.float64))
        ny, nx = self.ny, self.nx
        cex, cexc = _full(self.cex, ny, nx), _full(self.cex_curl, ny, nx)
        cey, ceyc = _full(self.cey, ny, nx), _full(self.cey_curl, ny, nx)
        ci, cb, cc, ck, pc = pml_pack(self.pml_c, ny, nx)
        xi, xb, xc, xk, px = pml_pack(self.pml_x, ny, nx)
        keys = ("h_r", "e_r", "h_t", "e_t")
        dft = np.zeros((4, nx, 2))
        for q, key in enumerate(keys):
            dft[q, :, 0] = self.dft[key].real
            dft[q, :, 1] = self.dft[key].imag
        a = _Args(nx, ny, self.dx, self.ch_curl, self.js,
                  0 if self.inc.kind == SOURCE_NONE else 1, self.jr, self.jt,
                  int(threads or self.threads))
        rc = _load().tez_loop_run(
            ctypes.byref(a), ctypes.c_int64(steps), _ptr(self.hz), _ptr(self.ex), _ptr(self.ey),
            _ptr(cex), _ptr(cexc), _ptr(cey), _ptr(ceyc),
            _ptr(ci), _ptr(cb), _ptr(cc), _ptr(ck), _ptr(pc),
            _ptr(xi), _ptr(xb), _ptr(xc), _ptr(xk), _ptr(px),
            _ptr(e_inc), _ptr(h_inc), _ptr(ph_h), _ptr(ph_e), _ptr(dft))
        if rc != 0:
            raise ValueError(f"tez_loop_run rejected the grid (status {rc})")
        pml_unpack(self.pml_c, pc)
        pml_unpack(self.pml_x, px)
        for q, key in enumerate(keys):
            v = np.empty(nx, dtype=np.complex128)
            v.real, v.imag = dft[q, :, 0], dft[q, :, 1]
            self.dft[key] = v
        self.n += steps
        return self


def run_rt_tez_c(spec, steps=None, threads=None):
    """run_rt_tez of the numpy oracle with the leaf run advanced by the C
    loop (the one-column empty-domain run stays in numpy)."""
    steps = spec.steps if steps is None else steps
    leaf = TEzOracleC(spec).run(steps, threads)
    twin = empty_twin_tez(spec).run(steps)
    p_up, p_down = leaf.fluxes()
    _, p0 = twin.fluxes()
    p_inc = p0 * spec.nx
    R, T = p_up / p_inc, p_down / p_inc
    return dict(R=R, T=T, A=1.0 - R - T, p_up=p_up, p_down=p_down, p_inc=p_inc,
                leaf=leaf, twin=twin)
