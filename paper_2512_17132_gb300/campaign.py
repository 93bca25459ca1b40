"""Spectral sweeps over many independent runs (wavelengths, slices,
polarisations), the way the paper builds its spectra (Sec. 4: one run per
wavelength, slice and polarisation; slice results averaged, polarisations
averaged for unpolarised light). The runs of a sweep go through batches
(fdtd_batch_*, one polarisation per batch), tuned once, so they share the
GPU. This module only orchestrates: every run steps in libfdtd.so.
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


def slice_specs(spec, n_slices=5, align=4):
    """Cut a cross-section into n_slices strips along x (Sec. 4: the leaf image
    is divided into five segments side by side, each run independently with
    periodic lateral boundaries). Every strip but the last is a multiple of
    `align` columns wide (the blocked kernel wants nx % 4 == 0); the last
    takes the remainder. Returns [(spec, width), ...]."""
    nx = int(spec.nx)
    w = (nx // n_slices) // align * align
    if n_slices < 1 or w < 1:
        raise ValueError(f"cannot cut {nx} columns into {n_slices} strips of >= {align}")
    bounds = [k * w for k in range(n_slices)] + [nx]
    out = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        lab = np.ascontiguousarray(np.asarray(spec.labels)[:, a:b])
        out.append((spec.with_(nx=b - a, labels=lab), b - a))
    return out


def _plan(make_spec, wavelengths, n_slices, pols):
    specs, widths = [], None
    for lam in wavelengths:
        cut = slice_specs(make_spec(lam), n_slices)
        if widths is None:
            widths = np.array([w for _, w in cut], dtype=np.float64)
        for sp, _ in cut:
            for p in pols:
                specs.append(sp.with_(polarization=int(p)))
    return specs, widths


def _assemble(R, T, wavelengths, n_slices, pols, widths):
    shape = (len(wavelengths), n_slices, len(pols))
    R_runs, T_runs = np.asarray(R).reshape(shape), np.asarray(T).reshape(shape)
    wk = widths / widths.sum()
    R_pol = np.einsum("lsp,s->lp", R_runs, wk)
    T_pol = np.einsum("lsp,s->lp", T_runs, wk)
    Rm, Tm = R_pol.mean(axis=1), T_pol.mean(axis=1)
    return dict(wavelengths=np.array(wavelengths), R_runs=R_runs, T_runs=T_runs, R_pol=R_pol,
                T_pol=T_pol, R=Rm, T=Tm, A=1.0 - Rm - Tm, widths=widths, pols=tuple(pols))


def shard(n_runs, rank, world):
    """Indices of the runs a rank takes (round-robin): the runs of a
    campaign are independent problems, so ranks share nothing but the final
    R and T scalars."""
    return list(range(rank, n_runs, world))


def gather_runs(n_runs, idx, R_loc, T_loc, world):
    """R and T of all runs on every rank, from each rank's share: one sum
    over the ranks of arrays that hold a rank's values at its own indices
    (host tensors under gloo, device tensors under NCCL)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.zeros((2, n_runs), dtype=torch.float64)
    t[0, idx] = torch.as_tensor(np.asarray(R_loc, dtype=np.float64))
    t[1, idx] = torch.as_tensor(np.asarray(T_loc, dtype=np.float64))
    t = t.to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    t = t.cpu().numpy()
    return t[0], t[1]


def run_campaign(make_spec, wavelengths, n_slices=5, pols=(fdtd.FDTD_POL_S, fdtd.FDTD_POL_P),
                 steps=None, runner=None, chunk=64, rank=0, world=1):
    """Spectrum of a cross-section the way Sec. 4 builds it: for every
    wavelength, every slice and every polarisation one independent run; the
    slices are averaged (weighted by width, the plain mean for equal strips)
    and the polarisations averaged (unpolarised light, Sec. 2.1).

    make_spec(lambda0) -> the full-width RunSpec at that wavelength (its
    material table evaluated there). runner(specs, steps) -> (R, T) arrays;
    the default is run_sweep (batched, one batch per polarisation). Returns
    a dict: wavelengths; R_runs, T_runs of shape (n_lambda, n_slices, n_pols);
    R_pol, T_pol (n_lambda, n_pols) slice-averaged; R, T, A (n_lambda)
    averaged over the polarisations; widths. With world > 1 (one process
    per GPU, torch.distributed initialised) each rank runs its round-robin
    share of the runs and every rank returns the whole campaign."""
    runner = runner or (lambda specs, st: run_sweep(specs, steps=st, chunk=chunk))
    wl = list(wavelengths)
    specs, widths = _plan(make_spec, wl, n_slices, pols)
    if world > 1:
        idx = shard(len(specs), rank, world)
        R_loc, T_loc = runner([specs[i] for i in idx], steps) if idx else ([], [])
        R, T = gather_runs(len(specs), idx, R_loc, T_loc, world)
    else:
        R, T = runner(specs, steps)
    return _assemble(R, T, wl, n_slices, pols, widths)


class Campaign:
    """A campaign kept resident for repeated runs: one handle per (wavelength,
    slice, polarisation) and one tuned batch per polarisation (at most
    `chunk` handles each), created once. run(steps) resets every handle,
    advances the batches and returns the run_campaign result dict."""

    def __init__(self, make_spec, wavelengths, n_slices=5,
                 pols=(fdtd.FDTD_POL_S, fdtd.FDTD_POL_P), autotune=True, chunk=64, timing=False):
        self.wl, self.n_slices, self.pols = list(wavelengths), n_slices, tuple(pols)
        self.specs, self.widths = _plan(make_spec, self.wl, n_slices, self.pols)
        if any(sp.nx % 4 for sp in self.specs):
            raise ValueError("resident campaigns need slices with nx % 4 == 0")
        self.sims, self.batches = [], []
        try:
            self.sims = [fdtd.Simulation(sp, timing=timing) for sp in self.specs]
            for p in self.pols:
                idx = [i for i, sp in enumerate(self.specs) if sp.polarization == p]
                for lo in range(0, len(idx), chunk):
                    b = fdtd.Batch([self.sims[i] for i in idx[lo:lo + chunk]], timing=timing)
                    if autotune:
                        b.autotune(2)
                    self.batches.append(b)
        except Exception:
            self.close()
            raise

    @property
    def cell_updates_per_step(self):
        return sum(sp.nx * sp.ny for sp in self.specs)

    def run(self, steps):
        for s in self.sims:
            s.reset()
        for b in self.batches:
            b.run(steps)
        RT = np.array([s.flux() for s in self.sims])
        return _assemble(RT[:, 0], RT[:, 1], self.wl, self.n_slices, self.pols, self.widths)

    def stats(self):
        return [b.stats() for b in self.batches]

    def close(self):
        for b in self.batches:
            b.close()
        for s in self.sims:
            s.close()
        self.batches, self.sims = [], []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
