"""ctypes binding of libfdtd (include/fdtd.h): same names, argument
marshalling only. Every step of the FDTD path runs in the CUDA library; if
the library is missing this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# FDTD_LIB selects another build of the library (the debug build for the
# index-check tests); the default is the release build next to this file
LIB_PATH = os.environ.get("FDTD_LIB") or os.path.join(HERE, "libfdtd.so")

FDTD_OK, FDTD_EINVAL, FDTD_ENOMEM, FDTD_ECUDA = 0, -1, -2, -3
FDTD_EUNSTABLE, FDTD_EBOUNDS, FDTD_ESTATE = -4, -5, -6
FDTD_OPT_KERNEL, FDTD_OPT_BLOCK_STEPS, FDTD_OPT_SEG_ROWS = 1, 2, 3
FDTD_OPT_TIMING, FDTD_OPT_WATCHDOG, FDTD_OPT_VARIANT, FDTD_OPT_GRAPH = 4, 5, 6, 7
FDTD_OPT_PLAN_WEIGHT = 8
FDTD_OPT_DEBUG_TABLE_LIMIT, FDTD_OPT_DEBUG_POKE_GUARD = 9, 10
FDTD_OPT_ADJ_BLOCK = 11
FDTD_POL_S, FDTD_POL_P = 0, 1
KERNEL_AUTO, KERNEL_NAIVE, KERNEL_BLOCKED = 0, 1, 2


class fdtd_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("dx", C.c_double), ("dt", C.c_double),
                ("pml_cells", C.c_int32), ("tfsf_row", C.c_int32), ("r_row", C.c_int32),
                ("t_row", C.c_int32), ("pml_order", C.c_double), ("pml_sigma_max", C.c_double),
                ("pml_kappa_max", C.c_double), ("pml_alpha_max", C.c_double)]


class fdtd_material(C.Structure):
    _fields_ = [("n", C.c_double), ("k", C.c_double)]


class fdtd_source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("polarization", C.c_int32), ("lambda0", C.c_double),
                ("rel_bandwidth", C.c_double), ("t0_over_tau", C.c_double)]


class fdtd_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("stencil_launches", C.c_int64),
                ("total_launches", C.c_int64), ("stencil_ms", C.c_double),
                ("kernel", C.c_int32), ("block_steps", C.c_int32), ("seg_rows", C.c_int32),
                ("variant", C.c_int32), ("graph", C.c_int32)]


class FDTDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libfdtd error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfdtd.so (built by paper_2512_17132_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(
            f"{path} is missing: build it with paper_2512_17132_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
    sig = {
        "fdtd_create": (C.c_int, [C.POINTER(fdtd_grid), vp, C.POINTER(fdtd_material), i32,
                                  C.POINTER(fdtd_source), vp, C.POINTER(vp)]),
        "fdtd_run": (C.c_int, [vp, i64]),
        "fdtd_synchronize": (C.c_int, [vp]),
        "fdtd_reset": (C.c_int, [vp]),
        "fdtd_flux": (C.c_int, [vp, dp, dp]),
        "fdtd_flux_raw": (C.c_int, [vp, dp]),
        "fdtd_get_dft": (C.c_int, [vp, vp]),
        "fdtd_reset_dft": (C.c_int, [vp]),
        "fdtd_bloch_orders": (C.c_int, [vp, i32, vp]),
        "fdtd_bloch_propagating": (i32, [vp]),
        "fdtd_get_fields": (C.c_int, [vp, vp, vp, vp]),
        "fdtd_set_fields": (C.c_int, [vp, vp, vp, vp]),
        "fdtd_state_bytes": (C.c_size_t, [vp]),
        "fdtd_save_state": (C.c_int, [vp, vp, C.c_size_t]),
        "fdtd_load_state": (C.c_int, [vp, vp, C.c_size_t]),
        "fdtd_set_option": (C.c_int, [vp, i32, i64]),
        "fdtd_get_stats": (C.c_int, [vp, C.POINTER(fdtd_stats)]),
        "fdtd_last_error": (C.c_char_p, [vp]),
        "fdtd_destroy": (None, [vp]),
        "fdtd_create_maps": (C.c_int, [C.POINTER(fdtd_grid), vp, vp, C.POINTER(fdtd_source), vp,
                                       C.POINTER(vp)]),
        "fdtd_forward_checkpointed": (C.c_int, [vp, i64, i32]),
        "fdtd_backward": (C.c_int, [vp, C.c_double, C.c_double, vp, vp, vp, dp]),
        "fdtd_autotune": (C.c_int, [vp, i32]),
        "fdtd_plan_segments": (C.c_int, [C.POINTER(fdtd_grid), i32, i32, i32,
                                         C.POINTER(C.c_int32), i32]),
        "fdtd_batch_create": (C.c_int, [C.POINTER(vp), i32, C.POINTER(vp)]),
        "fdtd_batch_set_option": (C.c_int, [vp, i32, i64]),
        "fdtd_batch_autotune": (C.c_int, [vp, i32]),
        "fdtd_batch_run": (C.c_int, [vp, i64]),
        "fdtd_batch_get_stats": (C.c_int, [vp, C.POINTER(fdtd_stats)]),
        "fdtd_batch_last_error": (C.c_char_p, [vp]),
        "fdtd_batch_destroy": (None, [vp]),
        "fdtd_blocked_advance_noalloc": (C.c_int, [C.POINTER(fdtd_grid), vp,
                                                   C.POINTER(fdtd_material), i32, C.c_double,
                                                   C.POINTER(vp), C.POINTER(vp), i32, vp,
                                                   C.c_char_p, C.c_size_t]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code, h):
    if code != FDTD_OK:
        msg = load_library().fdtd_last_error(h)
        raise FDTDError(code, msg.decode() if msg else "")


def _ptr(x):
    """Device or host pointer of a numpy array or a torch tensor (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


def make_grid(spec) -> fdtd_grid:
    return fdtd_grid(int(spec.nx), int(spec.ny), float(spec.dx), float(spec.dt),
                     int(spec.pml_cells), int(spec.tfsf_row), int(spec.r_row), int(spec.t_row),
                     float(spec.pml_order), float(spec.pml_sigma_max),
                     float(spec.pml_kappa_max), float(spec.pml_alpha_max))


def make_source(spec) -> fdtd_source:
    """The source of a spec; spec.polarization (0 = S/TMz, 1 = P/TEz) defaults to S."""
    return fdtd_source(int(spec.source_kind), int(getattr(spec, "polarization", FDTD_POL_S)),
                       float(spec.lambda0),
                       float(spec.rel_bandwidth), float(spec.t0_over_tau))


def fdtd_create(grid: fdtd_grid, labels, materials, source: fdtd_source, stream=None):
    """labels: (ny, nx) uint8 numpy array (host) or torch uint8 tensor (device);
    materials: (n_labels, 2) array of (n, k). Returns an opaque handle."""
    lib = load_library()
    if not hasattr(labels, "data_ptr"):
        labels = np.ascontiguousarray(labels, dtype=np.uint8)
    mats = np.ascontiguousarray(materials, dtype=np.float64).reshape(-1, 2)
    table = (fdtd_material * len(mats))(*[fdtd_material(float(n), float(k)) for n, k in mats])
    out = C.c_void_p()
    st = C.c_void_p(stream) if isinstance(stream, int) else (
        C.c_void_p(stream.cuda_stream) if stream is not None else None)
    code = lib.fdtd_create(C.byref(grid), _ptr(labels), table, len(mats), C.byref(source), st,
                           C.byref(out))
    _check(code, None)
    return out


def fdtd_create_maps(grid: fdtd_grid, eps_r, sigma, source: fdtd_source, stream=None):
    """eps_r, sigma: (ny, nx) float64 numpy arrays or device tensors."""
    lib = load_library()
    if not hasattr(eps_r, "data_ptr"):
        eps_r = np.ascontiguousarray(eps_r, dtype=np.float64)
    if not hasattr(sigma, "data_ptr"):
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    out = C.c_void_p()
    st = C.c_void_p(stream) if isinstance(stream, int) else (
        C.c_void_p(stream.cuda_stream) if stream is not None else None)
    _check(lib.fdtd_create_maps(C.byref(grid), _ptr(eps_r), _ptr(sigma), C.byref(source), st,
                                C.byref(out)), None)
    return out


def fdtd_forward_checkpointed(h, steps: int, every: int):
    _check(load_library().fdtd_forward_checkpointed(h, int(steps), int(every)), h)


def fdtd_backward(h, wR: float, wT: float, ny: int, nx: int, n_labels: int = 0, out=None):
    """Returns dict(J, R, T, g_eps, g_sigma[, g_n, g_k]); `out` may hold
    (g_eps, g_sigma) device tensors to fill instead of host arrays."""
    if out is None:
        ge = np.empty((ny, nx), dtype=np.float64)
        gs = np.empty((ny, nx), dtype=np.float64)
    else:
        ge, gs = out
    gl = np.zeros(2 * n_labels, dtype=np.float64) if n_labels else None
    jrt = (C.c_double * 3)()
    _check(load_library().fdtd_backward(h, float(wR), float(wT), _ptr(ge), _ptr(gs),
                                        _ptr(gl), jrt), h)
    res = {"J": jrt[0], "R": jrt[1], "T": jrt[2], "g_eps": ge, "g_sigma": gs}
    if gl is not None:
        res["g_n"], res["g_k"] = gl[0::2].copy(), gl[1::2].copy()
    return res


def fdtd_run(h, steps: int):
    _check(load_library().fdtd_run(h, int(steps)), h)


def fdtd_reset(h):
    _check(load_library().fdtd_reset(h), h)


def fdtd_synchronize(h):
    _check(load_library().fdtd_synchronize(h), h)


def fdtd_flux(h):
    R, T = C.c_double(), C.c_double()
    _check(load_library().fdtd_flux(h, C.byref(R), C.byref(T)), h)
    return R.value, T.value


def fdtd_flux_raw(h):
    out = (C.c_double * 3)()
    _check(load_library().fdtd_flux_raw(h, out), h)
    return tuple(out)


def fdtd_get_dft(h, nx: int):
    out = np.empty(8 * nx, dtype=np.float64)
    _check(load_library().fdtd_get_dft(h, _ptr(out)), h)
    z = out.reshape(4, nx, 2)
    return z[..., 0] + 1j * z[..., 1]


def fdtd_reset_dft(h):
    _check(load_library().fdtd_reset_dft(h), h)


def fdtd_bloch_propagating(h) -> int:
    r = int(load_library().fdtd_bloch_propagating(h))
    _check(min(r, 0), h)
    return r


def fdtd_plan_segments(grid: fdtd_grid, seg_rows: int, block_steps: int,
                       polarization: int = FDTD_POL_S) -> np.ndarray:
    """Row boundaries of the blocked kernel's segment plan (host only)."""
    lib = load_library()
    cap = int(grid.ny) + 1
    out = (C.c_int32 * cap)()
    r = int(lib.fdtd_plan_segments(C.byref(grid), int(seg_rows), int(block_steps),
                                   int(polarization), out, cap))
    _check(min(r, 0), None)
    return np.frombuffer(out, dtype=np.int32, count=r).copy()


BLOCH_FIELDS = ("R_flux", "T_flux", "R_paper", "T_paper", "R_corr", "T_corr", "w", "ky")


def fdtd_bloch_orders(h, m_max: int):
    """Per-order quantities for m = -m_max..m_max as a dict of numpy arrays
    (keys "m" and BLOCH_FIELDS, in the order of the C interface)."""
    out = np.empty((max(2 * int(m_max) + 1, 1), 8), dtype=np.float64)
    _check(load_library().fdtd_bloch_orders(h, int(m_max), _ptr(out)), h)
    d = {k: out[:, q].copy() for q, k in enumerate(BLOCH_FIELDS)}
    d["m"] = np.arange(-m_max, m_max + 1)
    return d


def fdtd_get_fields(h, ny: int, nx: int, out=None):
    """Returns (ez, hx, hy) float32 SI arrays (host), or fills `out` tensors."""
    if out is None:
        out = tuple(np.empty((ny, nx), dtype=np.float32) for _ in range(3))
    _check(load_library().fdtd_get_fields(h, *[_ptr(x) for x in out]), h)
    return out


def fdtd_set_fields(h, ez=None, hx=None, hy=None):
    args = []
    for x in (ez, hx, hy):
        if x is not None and not hasattr(x, "data_ptr"):
            x = np.ascontiguousarray(x, dtype=np.float32)
        args.append(x)
    _check(load_library().fdtd_set_fields(h, *[_ptr(x) for x in args]), h)


def fdtd_state_bytes(h) -> int:
    return int(load_library().fdtd_state_bytes(h))


def fdtd_save_state(h, buf=None):
    n = fdtd_state_bytes(h)
    if buf is None:
        buf = np.empty(n, dtype=np.uint8)
    _check(load_library().fdtd_save_state(h, _ptr(buf), n), h)
    return buf


def fdtd_load_state(h, buf):
    n = buf.numel() if hasattr(buf, "numel") else buf.nbytes
    _check(load_library().fdtd_load_state(h, _ptr(buf), n), h)


def fdtd_set_option(h, option: int, value: int):
    _check(load_library().fdtd_set_option(h, int(option), int(value)), h)


def fdtd_get_stats(h) -> dict:
    st = fdtd_stats()
    _check(load_library().fdtd_get_stats(h, C.byref(st)), h)
    return {k: getattr(st, k) for k, _ in fdtd_stats._fields_ if k != "graph"}


def fdtd_last_error(h=None) -> str:
    m = load_library().fdtd_last_error(h)
    return m.decode() if m else ""


def fdtd_destroy(h):
    if h:
        load_library().fdtd_destroy(h)


def fdtd_autotune(h, trial_launches: int = 4):
    _check(load_library().fdtd_autotune(h, int(trial_launches)), h)


def _check_batch(code, b):
    if code != FDTD_OK:
        msg = load_library().fdtd_batch_last_error(b)
        raise FDTDError(code, msg.decode() if msg else "")


def fdtd_batch_create(handles):
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h
                                         for h in handles])
    out = C.c_void_p()
    _check_batch(load_library().fdtd_batch_create(arr, len(handles), C.byref(out)), None)
    return out


def fdtd_batch_set_option(b, option: int, value: int):
    _check_batch(load_library().fdtd_batch_set_option(b, int(option), int(value)), b)


def fdtd_batch_autotune(b, trial_launches: int = 4):
    _check_batch(load_library().fdtd_batch_autotune(b, int(trial_launches)), b)


def fdtd_batch_run(b, steps: int):
    _check_batch(load_library().fdtd_batch_run(b, int(steps)), b)


def fdtd_batch_get_stats(b) -> dict:
    st = fdtd_stats()
    _check_batch(load_library().fdtd_batch_get_stats(b, C.byref(st)), b)
    d = {k: getattr(st, k) for k, _ in fdtd_stats._fields_}
    d["graph"] = bool(st.graph)
    return d


def fdtd_batch_last_error(b=None) -> str:
    m = load_library().fdtd_batch_last_error(b)
    return m.decode() if m else ""


def fdtd_batch_destroy(b):
    if b:
        load_library().fdtd_batch_destroy(b)


class Batch:
    """Owner of one fdtd_batch over a list of Simulation objects."""

    def __init__(self, sims, timing=False, graph=True):
        self.sims = list(sims)
        self.b = fdtd_batch_create([s.h for s in self.sims])
        if timing:
            fdtd_batch_set_option(self.b, FDTD_OPT_TIMING, 1)
        if not graph:
            fdtd_batch_set_option(self.b, FDTD_OPT_GRAPH, 0)

    def autotune(self, trial_launches=4):
        fdtd_batch_autotune(self.b, trial_launches)
        return self

    def run(self, steps):
        fdtd_batch_run(self.b, steps)
        return self

    def stats(self):
        return fdtd_batch_get_stats(self.b)

    def close(self):
        if self.b:
            fdtd_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_noalloc_tensors(grid: fdtd_grid, labels, inputs, outputs):
    """Checks the caller's tensors before any launch: dtype, contiguity and
    size first, then that each lives on the current CUDA device, so a host
    tensor or a short buffer never reaches the kernel."""
    def bad(msg):
        raise FDTDError(FDTD_EINVAL, "fdtd_blocked_advance_noalloc: " + msg)

    import torch
    nx, ny, P = int(grid.nx), int(grid.ny), int(grid.pml_cells)
    if len(inputs) != 5 or len(outputs) != 5:
        bad("inputs and outputs are five tensors each")
    want = [ny * nx] * 3 + [2 * P * nx] * 2
    names = ("Ez", "eta0*Hx", "eta0*Hy", "psi_E", "psi_H")
    if not isinstance(labels, torch.Tensor) or labels.dtype != torch.uint8:
        bad("labels must be a uint8 tensor")
    if not labels.is_contiguous() or labels.numel() < ny * nx:
        bad(f"labels must be contiguous with at least {ny * nx} elements")
    for side, ts in (("input", inputs), ("output", outputs)):
        for t, n, nm in zip(ts, want, names):
            if not isinstance(t, torch.Tensor) or t.dtype != torch.float32:
                bad(f"{side} {nm} must be a float32 tensor")
            if not t.is_contiguous() or t.numel() < max(n, 1):
                bad(f"{side} {nm} must be contiguous with at least {n} elements")
    for t in (labels, *inputs, *outputs):
        if not t.is_cuda:
            bad("every tensor must be on a CUDA device")
        if t.device.index != torch.cuda.current_device():
            bad("every tensor must be on the current CUDA device")


def fdtd_blocked_advance_noalloc(grid: fdtd_grid, labels, materials, lambda0: float,
                                 inputs, outputs, steps: int, stream=None):
    """Allocation-free stepping (see include/fdtd.h): inputs/outputs are five
    device tensors each {Ez, eta0*Hx, eta0*Hy, psi_E, psi_H}; labels a device
    uint8 tensor. The tensors are checked first; raises FDTDError with the
    library's message on failure."""
    _check_noalloc_tensors(grid, labels, inputs, outputs)
    lib = load_library()
    mats = np.ascontiguousarray(materials, dtype=np.float64).reshape(-1, 2)
    table = (fdtd_material * len(mats))(*[fdtd_material(float(n), float(k)) for n, k in mats])
    ins = (C.c_void_p * 5)(*[x.data_ptr() for x in inputs])
    outs = (C.c_void_p * 5)(*[x.data_ptr() for x in outputs])
    st = C.c_void_p(stream) if isinstance(stream, int) else (
        C.c_void_p(stream.cuda_stream) if stream is not None else None)
    err = C.create_string_buffer(256)
    code = lib.fdtd_blocked_advance_noalloc(C.byref(grid), _ptr(labels), table, len(mats),
                                            float(lambda0), ins, outs, int(steps), st, err, 256)
    if code != FDTD_OK:
        raise FDTDError(code, err.value.decode())


class Simulation:
    """Convenience owner of one handle, built from a run spec (an object with
    the fields of fdtd_inputs.RunSpec)."""

    def __init__(self, spec, stream=None, kernel: int = KERNEL_AUTO, block_steps=None,
                 seg_rows=None, timing=False, labels=None, eps_r=None, sigma=None):
        self.spec = spec
        self._maps = eps_r is not None
        if eps_r is not None:
            self.h = fdtd_create_maps(make_grid(spec), eps_r, sigma, make_source(spec), stream)
        else:
            lab = spec.labels if labels is None else labels
            self.h = fdtd_create(make_grid(spec), lab, spec.materials, make_source(spec), stream)
        try:
            if kernel:
                fdtd_set_option(self.h, FDTD_OPT_KERNEL, kernel)
            if block_steps:
                fdtd_set_option(self.h, FDTD_OPT_BLOCK_STEPS, block_steps)
            if seg_rows:
                fdtd_set_option(self.h, FDTD_OPT_SEG_ROWS, seg_rows)
            if timing:
                fdtd_set_option(self.h, FDTD_OPT_TIMING, 1)
        except Exception:
            self.close()
            raise

    def run(self, steps):
        fdtd_run(self.h, steps)
        return self

    def reset(self):
        fdtd_reset(self.h)
        return self

    def gradient(self, steps, wR=1.0, wT=0.0, every=500):
        """Forward with checkpoints, then the discrete adjoint of wR R + wT T.
        The handle keeps the checkpoints and the backward pass's tape (about
        8 * every bytes per cell) for the next gradient; close() frees them."""
        fdtd_forward_checkpointed(self.h, steps, every)
        n_lab = 0 if getattr(self, "_maps", False) else len(self.spec.materials)
        return fdtd_backward(self.h, wR, wT, self.spec.ny, self.spec.nx, n_lab)

    def flux(self):
        return fdtd_flux(self.h)

    def flux_raw(self):
        return fdtd_flux_raw(self.h)

    def dft(self):
        return fdtd_get_dft(self.h, self.spec.nx)

    def reset_dft(self):
        fdtd_reset_dft(self.h)
        return self

    def bloch(self, m_max=None):
        """Bloch orders -m_max..m_max (default: every propagating order)."""
        if m_max is None:
            m_max = fdtd_bloch_propagating(self.h)
        return fdtd_bloch_orders(self.h, m_max)

    def fields(self):
        return fdtd_get_fields(self.h, self.spec.ny, self.spec.nx)

    def set_fields(self, ez=None, hx=None, hy=None):
        fdtd_set_fields(self.h, ez, hx, hy)

    def stats(self):
        return fdtd_get_stats(self.h)

    def close(self):
        if self.h:
            fdtd_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
