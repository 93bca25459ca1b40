"""Run specifications (grid, rows, source, CPML values, materials) of the workloads.

Every number here is an input value shared by the CUDA library and the oracle;
each side turns these values into update coefficients with its own code.

Physical constants follow the classical SI definitions used throughout:
c0 = 299 792 458 m/s, mu0 = 4 pi 1e-7 H/m, eps0 = 1/(mu0 c0^2), eta0 = mu0 c0.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

C0 = 299_792_458.0
MU0 = 4.0e-7 * math.pi
EPS0 = 1.0 / (MU0 * C0 * C0)
ETA0 = MU0 * C0

# Tissue labels of the leaf cross-sections (uint8 values of the label map).
LABELS = {
    "air": 0,
    "cuticle": 1,
    "wall": 2,
    "cytoplasm": 3,
    "vacuole": 4,
    "hypha": 5,
}

SOURCE_PULSE = 0   # Gaussian-modulated sinusoid
SOURCE_CW = 1      # raised-cosine-ramped sinusoid
SOURCE_NONE = 2    # no incident wave (fields come from an initial state)

POL_S = 0          # S polarisation: E along z (TMz)
POL_P = 1          # P polarisation: H along z (TEz)


@dataclasses.dataclass
class RunSpec:
    """One FDTD run: the grid, the row layout, the source and the label map.

    Rows are counted from the top (j = 0) downward, the propagation direction
    of the incident wave; columns are periodic.
    """

    name: str
    nx: int
    ny: int
    dx: float
    dt: float
    steps: int
    lambda0: float
    tfsf_row: int
    r_row: int
    t_row: int
    labels: np.ndarray            # (ny, nx) uint8, row-major
    materials: np.ndarray         # (n_labels, 2) float64: (n, kappa) per label
    pml_cells: int = 16
    pml_order: float = 3.0
    pml_sigma_max: float = 0.0
    pml_kappa_max: float = 1.0
    pml_alpha_max: float = 0.0
    source_kind: int = SOURCE_PULSE
    rel_bandwidth: float = 0.1
    t0_over_tau: float = 5.0
    polarization: int = POL_S     # POL_S: TMz (Ez, Hx, Hy); POL_P: TEz (Hz, Ex, Ey)

    @property
    def courant(self) -> float:
        return C0 * self.dt / self.dx

    @property
    def cell_updates(self) -> int:
        return self.nx * self.ny * self.steps

    def with_(self, **kw) -> "RunSpec":
        return dataclasses.replace(self, **kw)


def courant_dt(dx: float, courant: float = 0.5) -> float:
    """Time step for a Courant number S = c0 dt / dx."""
    return courant * dx / C0


def default_cpml(dx: float, lambda0: float, order: float = 3.0) -> dict:
    """CFS-CPML parameter values (Roden and Gedney's polynomial grading).

    sigma_max = 0.8 (m + 1) / (eta0 dx), kappa_max = 1,
    alpha_max = 0.05 * 2 pi f0 * eps0 with f0 = c0 / lambda0.
    """
    return dict(
        pml_order=order,
        pml_sigma_max=0.8 * (order + 1.0) / (ETA0 * dx),
        pml_kappa_max=1.0,
        pml_alpha_max=0.05 * 2.0 * math.pi * (C0 / lambda0) * EPS0,
    )


def leaf_materials(lambda_m: float, n_labels: int = 6) -> np.ndarray:
    """(n, kappa) per leaf label at wavelength lambda (metres).

    Cuticle n = 1.45 and cell wall n = 1.52 follow Sec. 2.8; cytoplasm,
    vacuole and the melanised hypha use closed-form kappa(lambda) curves that
    stand in for the pigment, water and melanin data of Sec. 2.8 and Sec. 4.2.
    """
    lam = lambda_m * 1e9
    k_cyt = 0.02 * (math.exp(-((lam - 430.0) / 25.0) ** 2)
                    + 0.8 * math.exp(-((lam - 662.0) / 20.0) ** 2))
    k_vac = (1e-4 * math.exp(-((lam - 1450.0) / 50.0) ** 2)
             + 1e-3 * math.exp(-((lam - 1940.0) / 60.0) ** 2))
    k_hyp = 0.1 * (550.0 / lam) ** 2
    table = np.array([
        [1.0, 0.0],       # air
        [1.45, 0.0],      # cuticle
        [1.52, 0.0],      # cell wall
        [1.40, k_cyt],    # cytoplasm (pigmented, incl. chloroplasts)
        [1.34, k_vac],    # vacuole (water)
        [1.70, k_hyp],    # melanised hypha
    ], dtype=np.float64)
    return table[:n_labels].copy()


# ---------------------------------------------------------------------------
# Config 1: 256 x 256 slab stack (dx = 20 nm, S = 0.5, 4000 steps, 550 nm).
# Rows: 0-15 CPML | 20 R monitor | 24 TF/SF | 40-89 cuticle (1 um)
#       | 90-214 slab (2.5 um, n = 1.42, kappa = 1e-3) | 230 T monitor | 240-255 CPML
# ---------------------------------------------------------------------------
C1_ROWS = dict(r_row=20, tfsf_row=24, cuticle=(40, 90), slab=(90, 215), t_row=230)


def c1_materials() -> np.ndarray:
    return np.array([[1.0, 0.0], [1.45, 0.0], [1.42, 1e-3], [2.0, 0.0]],
                    dtype=np.float64)


def _base(name, nx, ny, dx, steps, lambda0, rows, labels, materials, **kw):
    spec = RunSpec(
        name=name, nx=nx, ny=ny, dx=dx, dt=courant_dt(dx), steps=steps,
        lambda0=lambda0, tfsf_row=rows["tfsf_row"], r_row=rows["r_row"],
        t_row=rows["t_row"], labels=labels, materials=materials,
        **default_cpml(dx, lambda0))
    return spec.with_(**kw) if kw else spec


def config_c1(nx: int = 256, steps: int = 4000, **kw) -> RunSpec:
    """Config 1: air / 1 um cuticle / 2.5 um lossy slab / air, x-uniform."""
    from .geometry import c1_labels
    labels = c1_labels(nx)
    return _base("c1", nx, 256, 20e-9, steps, 550e-9, C1_ROWS, labels,
                 c1_materials()[:3], **kw)


def config_c1b(nx: int = 256, steps: int = 4000, seed: int = 1, **kw) -> RunSpec:
    """Config 1b: config 1 plus four n = 2 cylinders and 1 % label noise."""
    from .geometry import c1b_labels
    labels = c1b_labels(nx, seed=seed)
    return _base("c1b", nx, 256, 20e-9, steps, 550e-9, C1_ROWS, labels,
                 c1_materials(), **kw)


def dicot_rows(ny: int, dx: float) -> dict:
    """Row layout of a dicot cross-section that fits a domain of ny rows.

    Layer thicknesses (um): cuticle 2, upper epidermis 12, palisade 40,
    spongy 74, lower epidermis 12 (140 um in total); they shrink in proportion
    when the domain is shorter than the leaf plus its margins.
    """
    per_um = 1e-6 / dx
    top = 100
    rows_avail = ny - 16 - top - 150
    scale = min(1.0, rows_avail / (140.0 * per_um))
    thick = [2.0, 12.0, 40.0, 74.0, 12.0]
    edges = [top]
    for t in thick:
        edges.append(edges[-1] + max(2, int(round(t * per_um * scale))))
    leaf_bottom = edges[-1]
    return dict(r_row=40, tfsf_row=60, layer_edges=edges,
                t_row=min(leaf_bottom + 100, ny - 16 - 4))


def config_c2(lambda0: float = 550e-9, seed: int = 0, steps: int = 30000,
              nx: int = 2000, ny: int = 12500, labels: Optional[np.ndarray] = None,
              **kw) -> RunSpec:
    """Config 2: 40 um x 250 um dicot cross-section at dx = 20 nm."""
    from .geometry import dicot_labels
    dx = 20e-9
    rows = dicot_rows(ny, dx)
    if labels is None:
        labels = dicot_labels(nx, ny, dx, rows, seed=seed)
    return _base("c2", nx, ny, dx, steps, lambda0, rows, labels,
                 leaf_materials(lambda0), **kw)


C2_WAVELENGTHS = (450e-9, 550e-9, 662e-9, 800e-9, 1450e-9)


def monocot_rows(ny: int, dx: float) -> dict:
    """Row layout of the monocot cross-section (cuticle 2 um, epidermis 12 um,
    mesophyll 80 um, lower epidermis 12 um, lower cuticle 1 um)."""
    per_um = 1e-6 / dx
    top = 100
    thick = [2.0, 12.0, 80.0, 12.0, 1.0]
    rows_avail = ny - 16 - top - 150
    scale = min(1.0, rows_avail / (sum(thick) * per_um))
    edges = [top]
    for t in thick:
        edges.append(edges[-1] + max(2, int(round(t * per_um * scale))))
    return dict(r_row=40, tfsf_row=60, layer_edges=edges,
                t_row=min(edges[-1] + int(round(2.0 * per_um)), ny - 16 - 4))


def config_c3(lambda0: float = 550e-9, diseased: bool = False, seed: int = 0,
              steps: int = 60000, nx: int = 8192, ny: int = 32768,
              labels: Optional[np.ndarray] = None, **kw) -> RunSpec:
    """Config 3: 123 um x 492 um monocot cross-section at dx = 15 nm,
    optionally with 12 melanised hyphae."""
    from .geometry import monocot_labels
    dx = 15e-9
    rows = monocot_rows(ny, dx)
    if labels is None:
        labels = monocot_labels(nx, ny, dx, rows, seed=seed,
                                n_hyphae=12 if diseased else 0)
    return _base("c3" + ("-diseased" if diseased else ""), nx, ny, dx, steps,
                 lambda0, rows, labels, leaf_materials(lambda0), **kw)


def _c4_labels(job):
    """Label map of one config-4 simulation (a top-level function, so that a
    process pool can run it)."""
    from .geometry import dicot_labels
    nx, ny, dx, rows, seed, n_hyphae, coarse = job
    return dicot_labels(nx, ny, dx, rows, seed=seed, n_hyphae=n_hyphae, coarse=coarse)


def config_c4(n_sims: int = 64, seed: int = 0, steps: int = 30000,
              nx: int = 2000, height_range=(2000, 12500), coarse: int = 1,
              workers: Optional[int] = None) -> list:
    """Config 4: independent dicot simulations of uneven height.

    Heights are uniform in height_range (rounded to 4 rows), wavelengths lie on
    a 400-2500 nm grid shuffled by the seed, even indices are healthy and odd
    indices carry hyphae. Label maps are drawn at the grid's own resolution
    (coarse = 1); coarse > 1 draws them that many times coarser and repeats
    each cell (the layer edges rounded to multiples of `coarse`). With
    workers > 1 the maps are drawn in a process pool (spawned processes, safe
    after CUDA has been initialised in the caller).
    """
    rng = np.random.default_rng(seed)
    heights = (rng.integers(height_range[0], height_range[1] + 1, n_sims) // 4) * 4
    lams = 400e-9 + np.arange(n_sims) * (2100e-9 / max(1, n_sims - 1))
    lams = rng.permutation(lams)
    dx = 20e-9
    jobs, rows_all = [], []
    for i in range(n_sims):
        ny = int(heights[i])
        rows = dicot_rows(ny, dx)
        if coarse > 1:
            rows["layer_edges"] = [e // coarse * coarse for e in rows["layer_edges"]]
        rows_all.append(rows)
        jobs.append((nx, ny, dx, rows, 1000 + i, 3 if i % 2 else 0, coarse))
    if workers and workers > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            labels = list(ex.map(_c4_labels, jobs))
    else:
        labels = [_c4_labels(j) for j in jobs]
    return [_base(f"c4-{i}", nx, int(heights[i]), dx, steps, float(lams[i]), rows_all[i],
                  labels[i], leaf_materials(float(lams[i]))) for i in range(n_sims)]


def config_c5(steps: int = 30000, nx: int = 1000, ny: int = 6000,
              lambda0: float = 550e-9, **kw) -> RunSpec:
    """Config 5: the config-1 stack with physical thicknesses kept, extended
    to ny rows of air below, at 1000 columns (adjoint workload)."""
    from .geometry import stack_labels
    rows = dict(r_row=20, tfsf_row=24, t_row=230)
    labels = stack_labels(nx, ny, [(40, 90, 1), (90, 215, 2)])
    return _base("c5", nx, ny, 20e-9, steps, lambda0, rows, labels,
                 c1_materials()[:3], **kw)


def crop_layout(spec: RunSpec, ny: int, nx: Optional[int] = None) -> RunSpec:
    """Keep the first ny rows (and nx columns) of a spec: a smaller case of the
    same layout for tests; rows below the crop are dropped."""
    nx = spec.nx if nx is None else nx
    labels = np.ascontiguousarray(spec.labels[:ny, :nx])
    t_row = min(spec.t_row, ny - spec.pml_cells - 4)
    return spec.with_(nx=nx, ny=ny, labels=labels, t_row=t_row)


def config_e2(l_over_lambda: float, steps: int = 40000, nx: int = 100, ny: int = 897,
              pml_cells: int = 40, rel_bandwidth: float = 0.1, h: float = 0.01,
              diameter: float = 0.3, n_cyl: float = 2.0) -> RunSpec:
    """Validation workload of Sec. 3: a periodic array of dielectric cylinders
    (period L = 1 m = 100 cells at h = 0.01 m, diameter D = 0.3 m, n = 2)
    under a normally incident S-polarised (TMz) wave, dt = 23.57 ps (Sec. 3
    table). The paper's unit cell is periodic in y with PML in x; here the
    same cell is periodic in x with the CPML at top and bottom (axes
    rotated). A finer cell h < 0.01 m scales the cell counts, the CPML
    thickness and dt by 0.01 / h (the same Courant number, the same physical
    domain); pass steps scaled alike for the same physical run time.
    diameter (m) and n_cyl vary the cylinder for sensitivity studies."""
    from .geometry import cylinder_array_labels
    f = 0.01 / h
    if f != 1.0:
        nx, ny, pml_cells = int(round(nx * f)), int(round(ny * f)), int(round(pml_cells * f))
    dx = h
    lam = 1.0 / l_over_lambda
    rows = dict(r_row=pml_cells + int(round(10 * f)), tfsf_row=pml_cells + int(round(20 * f)),
                t_row=ny - pml_cells - int(round(12 * f)))
    labels = cylinder_array_labels(nx, ny, radius_cells=0.5 * diameter / h)
    mats = np.array([[1.0, 0.0], [n_cyl, 0.0]])
    spec = _base("e2", nx, ny, dx, steps, lam, rows, labels, mats, pml_cells=pml_cells,
                 rel_bandwidth=rel_bandwidth)
    return spec.with_(dt=23.57e-12 * h / 0.01)
