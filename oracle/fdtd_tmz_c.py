"""The TMz oracle with its time loop in plain C (oracle/tmz_loop.c).

TEST INFRASTRUCTURE, like the rest of this package. TMzOracleC is the numpy
oracle (fdtd_tmz.TMzOracle: same constructor, state, coefficients, CPML
profiles, incident line, DFT phases and fluxes); only run(steps) hands the
leapfrog loop to the C function, which repeats the numpy oracle's arithmetic
operation for operation, cell by cell, on all host cores. The two agree bit
for bit (tests/test_oracle_c.py), so every pin of the numpy oracle carries
over, and full-size grids finish in minutes per thousand steps instead of
hours. The adjoint tape is recorded by the numpy loop only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .fdtd_tmz import SOURCE_NONE, TMzOracle, empty_twin

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tmz_loop.c")
LIB = os.path.join(HERE, "_tmz_loop.so")


def compile_loop(src: str, lib: str, force: bool = False) -> str:
    """Compile one C time loop with gcc (OpenMP, no FP contraction so that
    every product and sum rounds exactly as in numpy)."""
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, src]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"gcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


def pml_pack(layers, ny, nx):
    """The oracle's CPML layers ((rows, b, c, kappa, psi) per side) as the C
    loops take them: a row -> CPML-row index map (-1 outside), the per-row
    b, c, kappa and the psi rows stacked."""
    idx = np.full(ny, -1, dtype=np.int32)
    rows = [r for lay in layers for r in lay[0]]
    idx[np.asarray(rows, dtype=np.int64)] = np.arange(len(rows), dtype=np.int32)
    b = np.ascontiguousarray(np.concatenate([lay[1][:, 0] for lay in layers])) if rows else np.zeros(1)
    c = np.ascontiguousarray(np.concatenate([lay[2][:, 0] for lay in layers])) if rows else np.zeros(1)
    k = np.ascontiguousarray(np.concatenate([lay[3][:, 0] for lay in layers])) if rows else np.zeros(1)
    psi = (np.ascontiguousarray(np.concatenate([lay[4] for lay in layers]))
           if rows else np.zeros((1, nx)))
    return idx, b, c, k, psi


def pml_unpack(layers, psi):
    """Copy the stacked psi rows back into the oracle's layers."""
    o = 0
    for lay in layers:
        m = len(lay[0])
        lay[4][...] = psi[o:o + m]
        o += m


class _Args(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_double),
                ("ch_curl", ctypes.c_double), ("js", ctypes.c_int32), ("tfsf", ctypes.c_int32),
                ("jr", ctypes.c_int32), ("jt", ctypes.c_int32), ("threads", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the TMz C loop."""
    return compile_loop(SRC, LIB, force)


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.tmz_loop_run.restype = ctypes.c_int
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class TMzOracleC(TMzOracle):
    """TMzOracle whose run(steps) advances with the C loop."""

    threads = os.cpu_count() or 1

    def run(self, steps, threads=None):
        steps = int(steps)
        if steps <= 0:
            return self
        if self.tape is not None:
            raise RuntimeError("the adjoint tape is recorded by the numpy loop (TMzOracle)")
        # incident samples and DFT phases, taken exactly as TMzOracle.step() takes them
        h_inc = np.empty(steps)
        e_inc = np.empty(steps)
        ph_e = np.empty(2 * steps)
        ph_h = np.empty(2 * steps)
        for m in range(steps):
            n = self.n + m
            h_inc[m] = self.inc.h_inc()
            self.inc.advance_e()
            e_inc[m] = self.inc.e_inc()
            self.inc.advance_h()
            pe = np.exp(1j * self.omega * ((n + 0.5) * self.dt))
            ph = np.exp(1j * self.omega * ((n + 1.0) * self.dt))
            ph_e[2 * m], ph_e[2 * m + 1] = pe.real, pe.imag
            ph_h[2 * m], ph_h[2 * m + 1] = ph.real, ph.imag
        for name in ("ez", "hx", "hy"):
            setattr(self, name, np.ascontiguousarray(getattr(self, name), dtype=np.float64))
        ce = np.ascontiguousarray(np.broadcast_to(self.ce, (self.ny, self.nx)), dtype=np.float64)
        cc = np.ascontiguousarray(np.broadcast_to(self.ce_curl, (self.ny, self.nx)),
                                  dtype=np.float64)
        ei, eb, ec, ek, pe_ = pml_pack(self.pml_e, self.ny, self.nx)
        hi, hb, hc, hk, ph_ = pml_pack(self.pml_h, self.ny, self.nx)
        dft = np.zeros((4, self.nx, 2))
        for q, key in enumerate(("e_r", "h_r", "e_t", "h_t")):
            dft[q, :, 0] = self.dft[key].real
            dft[q, :, 1] = self.dft[key].imag
        a = _Args(self.nx, self.ny, self.dx, self.ch_curl, self.js,
                  0 if self.inc.kind == SOURCE_NONE else 1, self.jr, self.jt,
                  int(threads or self.threads))
        rc = _load().tmz_loop_run(
            ctypes.byref(a), ctypes.c_int64(steps), _ptr(self.ez), _ptr(self.hx), _ptr(self.hy),
            _ptr(ce), _ptr(cc), _ptr(ei), _ptr(eb), _ptr(ec), _ptr(ek), _ptr(pe_),
            _ptr(hi), _ptr(hb), _ptr(hc), _ptr(hk), _ptr(ph_),
            _ptr(h_inc), _ptr(e_inc), _ptr(ph_e), _ptr(ph_h), _ptr(dft))
        if rc != 0:
            raise ValueError(f"tmz_loop_run rejected the grid (status {rc})")
        pml_unpack(self.pml_e, pe_)
        pml_unpack(self.pml_h, ph_)
        for q, key in enumerate(("e_r", "h_r", "e_t", "h_t")):
            v = np.empty(self.nx, dtype=np.complex128)
            v.real, v.imag = dft[q, :, 0], dft[q, :, 1]
            self.dft[key] = v
        self.n += steps
        return self


def run_rt_c(spec, steps=None, threads=None):
    """run_rt of the numpy oracle with both runs (leaf and empty domain)
    advanced by the C loop."""
    steps = spec.steps if steps is None else steps
    leaf = TMzOracleC(spec).run(steps, threads)
    twin = empty_twin(spec).run(steps)
    p_up, p_down = leaf.fluxes()
    _, p0 = twin.fluxes()
    p_inc = p0 * spec.nx
    R, T = p_up / p_inc, p_down / p_inc
    return dict(R=R, T=T, A=1.0 - R - T, p_up=p_up, p_down=p_down, p_inc=p_inc,
                leaf=leaf, twin=twin)
