"""Seeded label maps (segmented cross-sections) for the workloads.

The paper builds its label maps from hand-segmented micrographs with randomly
inserted chloroplast ellipses (Sec. 2.7). The micrographs are not available,
so these generators draw synthetic tissue of the same kind from a seed:
layered cuticle / epidermis / palisade / spongy mesophyll with 0.3 um cell
walls, a 1 um cytoplasm lining, vacuoles, chloroplast ellipses sampled as in
Sec. 2.7 (a = 0.8 + 0.2 (2 r1 - 1) um, b = a (1 + (r2 - 0.5)), theta uniform),
and optional melanised hyphae (Sec. 4.2). All maps are uint8, shape (ny, nx),
row 0 at the top, periodic in x.
"""
from __future__ import annotations

import math

import numpy as np

from .configs import LABELS, C1_ROWS

AIR = LABELS["air"]
CUTICLE = LABELS["cuticle"]
WALL = LABELS["wall"]
CYTO = LABELS["cytoplasm"]
VAC = LABELS["vacuole"]
HYPHA = LABELS["hypha"]


def stack_labels(nx: int, ny: int, layers) -> np.ndarray:
    """x-uniform stack: layers = [(row_begin, row_end, label), ...]."""
    lab = np.zeros((ny, nx), dtype=np.uint8)
    for r0, r1, v in layers:
        lab[r0:r1, :] = v
    return lab


def cylinder_array_labels(nx: int, ny: int, radius_cells: float) -> np.ndarray:
    """One period of a cylinder array: a disc of label 1 centred in the
    middle row of a periodic strip of nx columns."""
    jj, ii = np.mgrid[0:ny, 0:nx]
    inside = (ii + 0.5 - nx / 2.0) ** 2 + (jj + 0.5 - ny / 2.0) ** 2 <= radius_cells ** 2
    return inside.astype(np.uint8)


def c1_labels(nx: int = 256) -> np.ndarray:
    """Config 1: air / cuticle rows 40-89 (label 1) / slab rows 90-214 (label 2)."""
    return stack_labels(nx, 256, [(*C1_ROWS["cuticle"], 1), (*C1_ROWS["slab"], 2)])


def c1b_labels(nx: int = 256, seed: int = 1, noise: float = 0.01) -> np.ndarray:
    """Config 1b: config 1 plus a periodic row of four D = 1 um (50 cell) n = 2
    cylinders (label 3) centred in the slab, and 1 % of the cells in rows
    40-214 (fraction `noise`) relabelled at random among labels 1-3."""
    lab = c1_labels(nx)
    rng = np.random.default_rng(seed)
    jj, ii = np.mgrid[0:256, 0:nx]
    yc = 0.5 * (C1_ROWS["slab"][0] + C1_ROWS["slab"][1])
    period = nx / 4.0
    for k in range(4):
        xc = (k + 0.5) * period
        dxw = (ii + 0.5 - xc + nx / 2.0) % nx - nx / 2.0
        inside = dxw ** 2 + (jj + 0.5 - yc) ** 2 <= 25.0 ** 2
        lab[inside] = 3
    r0, r1 = C1_ROWS["cuticle"][0], C1_ROWS["slab"][1]
    region = lab[r0:r1]
    mask = rng.random(region.shape) < noise
    region[mask] = rng.integers(1, 4, int(mask.sum()), dtype=np.uint8)
    return lab


# --------------------------------------------------------------------------
# Leaf tissue helpers
# --------------------------------------------------------------------------

def _cell_interior(lab, d, t_wall, t_cyto):
    """Label cell interiors by the distance d (cells) to the cell boundary:
    wall within t_wall, then a cytoplasm lining of t_cyto, then vacuole."""
    out = np.full(d.shape, VAC, dtype=np.uint8)
    out[d < t_wall + t_cyto] = CYTO
    out[d < t_wall] = WALL
    return out


def _ellipse_band(nx, r0, r1, ellipses, t_wall, t_cyto, background):
    """Rasterise a band of rows [r0, r1) holding axis-aligned ellipse cells.

    ellipses: list of (xc, yc, a, b) in cell units (yc absolute row). Each
    point takes the ellipse it lies deepest in; depth is the first-order
    distance estimate (1 - rho^2) / |grad rho^2|. Returns (labels, depth)."""
    jj, ii = np.mgrid[r0:r1, 0:nx].astype(np.float64)
    x = ii + 0.5
    y = jj + 0.5
    best = np.full(x.shape, -np.inf)
    for xc, yc, a, b in ellipses:
        dxw = (x - xc + nx / 2.0) % nx - nx / 2.0
        dy = y - yc
        g = (dxw / a) ** 2 + (dy / b) ** 2
        grad = 2.0 * np.sqrt((dxw / a ** 2) ** 2 + (dy / b ** 2) ** 2) + 1e-12
        depth = (1.0 - g) / grad
        np.maximum(best, depth, out=best)
    lab = _cell_interior(None, best, t_wall, t_cyto)
    lab[best < 0] = background
    return lab, best


def _voronoi_band(nx, r0, r1, seeds, shrink, t_wall, t_cyto, band_edge_wall=True):
    """Rasterise rows [r0, r1) as Voronoi cells (periodic in x) scaled about
    their seeds by `shrink` (area fraction shrink^2; the rest is air).

    A point x with nearest seed s1 lies in the shrunk cell iff the point
    s1 + (x - s1)/shrink has s1 as nearest seed too; its wall distance is
    shrink times the bisector distance of that point. Returns (labels, depth).
    """
    from scipy.spatial import cKDTree

    seeds = np.asarray(seeds, dtype=np.float64)
    ns = len(seeds)
    rep = np.concatenate([seeds - [nx, 0], seeds, seeds + [nx, 0]])
    tree = cKDTree(rep)
    lab = np.empty((r1 - r0, nx), dtype=np.uint8)
    dep = np.empty((r1 - r0, nx), dtype=np.float32)
    chunk = max(1, 2_000_000 // nx)
    xs = np.arange(nx, dtype=np.float64) + 0.5
    for c0 in range(r0, r1, chunk):
        c1 = min(r1, c0 + chunk)
        yy, xx = np.meshgrid(np.arange(c0, c1) + 0.5, xs, indexing="ij")
        pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
        _, i1 = tree.query(pts, k=1)
        s1 = rep[i1]
        q = s1 + (pts - s1) / shrink
        _, i2 = tree.query(q, k=2)
        inside = (i2[:, 0] % ns) == (i1 % ns)
        a = rep[i2[:, 0]]
        b = rep[i2[:, 1]]
        num = ((q - b) ** 2).sum(1) - ((q - a) ** 2).sum(1)
        den = 2.0 * np.sqrt(((b - a) ** 2).sum(1)) + 1e-12
        d = shrink * num / den
        if band_edge_wall:
            d = np.minimum(d, np.minimum(pts[:, 1] - r0, r1 - pts[:, 1]))
        out = _cell_interior(None, d, t_wall, t_cyto)
        out[~inside] = AIR
        d[~inside] = -1.0
        lab[c0 - r0:c1 - r0] = out.reshape(c1 - c0, nx)
        dep[c0 - r0:c1 - r0] = d.reshape(c1 - c0, nx)
    return lab, dep


def _jittered_seeds(rng, nx, r0, r1, spacing_x, spacing_y, jitter=0.35):
    """Seeds on a jittered lattice covering rows [r0, r1) (cell units)."""
    nxs = max(1, int(round(nx / spacing_x)))
    nys = max(1, int(round((r1 - r0) / spacing_y)))
    sx = nx / nxs
    sy = (r1 - r0) / nys
    seeds = []
    for q in range(nys):
        for p in range(nxs):
            off = 0.5 * sx if (q % 2) else 0.0
            seeds.append([((p + 0.5) * sx + off + rng.uniform(-jitter, jitter) * sx) % nx,
                          r0 + (q + 0.5) * sy + rng.uniform(-jitter, jitter) * sy])
    return np.array(seeds)


def _add_chloroplasts(rng, lab, depth, r0, r1, per_um, frac=0.2, l_chl_um=2.0,
                      t_wall=0.0):
    """Insert rotated chloroplast ellipses (Sec. 2.7) labelled cytoplasm into the
    cell interiors of rows [r0, r1) until they cover `frac` of the non-air
    mesophyll area; centres lie within l_chl of a cell wall."""
    ny_b, nx = r1 - r0, lab.shape[1]
    band = lab[r0:r1]
    cell_area = int((band != AIR).sum())
    target = frac * cell_area
    cand = np.flatnonzero(((band == VAC) | (band == CYTO)).ravel()
                          & (depth.ravel() < t_wall + l_chl_um * per_um))
    if len(cand) == 0:
        return
    covered = 0.0
    guard = 0
    while covered < target and guard < 200000:
        guard += 1
        r1_, r2_ = rng.random(2)
        a = (0.8 + 0.2 * (2.0 * r1_ - 1.0)) * per_um
        b = a * (1.0 + (r2_ - 0.5))
        th = rng.uniform(0.0, 2.0 * math.pi)
        p = cand[rng.integers(len(cand))]
        yc, xc = divmod(int(p), nx)
        R = int(math.ceil(max(a, b))) + 1
        y0, y1 = max(0, yc - R), min(ny_b, yc + R + 1)
        yy, xx = np.mgrid[y0:y1, xc - R:xc + R + 1]
        u = (xx - xc) * math.cos(th) + (yy - yc) * math.sin(th)
        v = -(xx - xc) * math.sin(th) + (yy - yc) * math.cos(th)
        ins = (u / a) ** 2 + (v / b) ** 2 <= 1.0
        xw = xx % nx
        sub = band[yy[ins], xw[ins]]
        ok = (sub == VAC) | (sub == CYTO)
        band[yy[ins][ok], xw[ins][ok]] = CYTO
        covered += float(ok.sum())


def _add_hyphae(rng, lab, top_row, per_um, n):
    """Vertical melanised hyphae: width U[2, 5] um, reaching U[10, 20] um below
    the leaf surface, with a semicircular tip (label HYPHA)."""
    ny, nx = lab.shape
    for _ in range(n):
        w = rng.uniform(2.0, 5.0) * per_um
        depth = rng.uniform(10.0, 20.0) * per_um
        xc = rng.uniform(0, nx)
        rad = 0.5 * w
        y_end = top_row + depth
        r0 = max(0, top_row - int(rad))
        r1 = min(ny, int(math.ceil(y_end + rad)) + 1)
        jj, ii = np.mgrid[r0:r1, 0:nx].astype(np.float64)
        dxw = (ii + 0.5 - xc + nx / 2.0) % nx - nx / 2.0
        y = jj + 0.5
        body = (np.abs(dxw) <= rad) & (y >= top_row) & (y <= y_end)
        tip = (dxw ** 2 + (y - y_end) ** 2) <= rad ** 2
        sel = body | tip
        lab[r0:r1][sel] = HYPHA


def dicot_labels(nx: int, ny: int, dx: float, rows: dict, seed: int = 0,
                 n_hyphae: int = 0, coarse: int = 1) -> np.ndarray:
    """Dicot-like cross-section: cuticle, an upper epidermis of 15 x 12 um
    ellipse cells, palisade columns of 10 x 40 um ellipses, spongy mesophyll of
    Voronoi cells shrunk to a 40 % air fraction, a lower epidermis, with
    0.3 um walls, 1 um cytoplasm linings and chloroplasts in the mesophyll.
    coarse > 1 draws the map on a grid `coarse` times coarser and repeats each
    cell (faster for large batches; nx, ny and the layer edges must divide)."""
    if coarse > 1:
        rc = dict(rows, layer_edges=[e // coarse for e in rows["layer_edges"]])
        small = dicot_labels(nx // coarse, ny // coarse, dx * coarse, rc, seed=seed,
                             n_hyphae=n_hyphae)
        return np.ascontiguousarray(np.repeat(np.repeat(small, coarse, 0), coarse, 1))
    rng = np.random.default_rng(seed)
    per_um = 1e-6 / dx
    e = rows["layer_edges"]
    scale = (e[-1] - e[0]) / (140.0 * per_um)
    t_wall = max(1.0, 0.3 * per_um)
    t_cyto = max(1.0, 1.0 * per_um * min(1.0, scale))
    lab = np.zeros((ny, nx), dtype=np.uint8)
    lab[e[0]:e[1]] = CUTICLE

    def epidermis(r0, r1):
        n = max(1, int(round(nx / (15.0 * per_um * max(scale, 0.2)))))
        h = r1 - r0
        ell = [((k + 0.5 + rng.uniform(-0.1, 0.1)) * nx / n, r0 + 0.5 * h,
                0.55 * nx / n, 0.5 * h) for k in range(n)]
        band, _ = _ellipse_band(nx, r0, r1, ell, t_wall, t_cyto, WALL)
        lab[r0:r1] = band

    epidermis(e[1], e[2])
    # palisade: one row of columnar ellipses (10 um wide)
    r0, r1 = e[2], e[3]
    n = max(1, int(round(nx / (10.0 * per_um * max(scale, 0.2)))))
    ell = [((k + 0.5 + rng.uniform(-0.08, 0.08)) * nx / n, 0.5 * (r0 + r1),
            0.46 * nx / n, 0.48 * (r1 - r0)) for k in range(n)]
    band, dep_p = _ellipse_band(nx, r0, r1, ell, t_wall, t_cyto, AIR)
    lab[r0:r1] = band
    # spongy: Voronoi cells (~12 um) shrunk to 60 % area
    r0s, r1s = e[3], e[4]
    sp = 12.0 * per_um * max(scale, 0.2)
    seeds = _jittered_seeds(rng, nx, r0s, r1s, sp, sp)
    band, dep_s = _voronoi_band(nx, r0s, r1s, seeds, math.sqrt(0.6), t_wall, t_cyto)
    lab[r0s:r1s] = band
    epidermis(e[4], e[5])
    dep = np.concatenate([dep_p.astype(np.float32), dep_s])
    _add_chloroplasts(rng, lab, dep, e[2], e[4], per_um * max(scale, 0.2),
                      t_wall=t_wall)
    if n_hyphae:
        _add_hyphae(rng, lab, e[0], per_um * max(scale, 0.2), n_hyphae)
    return lab


def monocot_labels(nx: int, ny: int, dx: float, rows: dict, seed: int = 0,
                   n_hyphae: int = 0) -> np.ndarray:
    """Monocot-like cross-section: cuticle, Voronoi epidermis, a uniform
    mesophyll of 8-14 um Voronoi cells with 25 % air and no palisade, lower
    epidermis and lower cuticle; optional melanised hyphae."""
    rng = np.random.default_rng(seed)
    per_um = 1e-6 / dx
    e = rows["layer_edges"]
    t_wall = max(1.0, 0.3 * per_um)
    t_cyto = 1.0 * per_um
    lab = np.zeros((ny, nx), dtype=np.uint8)
    lab[e[0]:e[1]] = CUTICLE
    for (r0, r1) in [(e[1], e[2]), (e[3], e[4])]:
        seeds = _jittered_seeds(rng, nx, r0, r1, 10.0 * per_um, (r1 - r0), 0.2)
        band, _ = _voronoi_band(nx, r0, r1, seeds, 1.0, t_wall, t_cyto)
        lab[r0:r1] = band
    r0, r1 = e[2], e[3]
    # seeds with spacing drawn from 8-14 um
    area = nx * (r1 - r0)
    mean_sp = 11.0 * per_um
    n_seeds = max(4, int(area / mean_sp ** 2))
    seeds = np.stack([rng.uniform(0, nx, n_seeds), rng.uniform(r0, r1, n_seeds)], 1)
    # one relaxation pass towards even spacing (sizes stay within ~8-14 um)
    from scipy.spatial import cKDTree
    for _ in range(3):
        tree = cKDTree(np.concatenate([seeds - [nx, 0], seeds, seeds + [nx, 0]]))
        d, idx = tree.query(seeds, k=2)
        nb = tree.data[idx[:, 1]]
        push = seeds - nb
        close = d[:, 1] < 8.0 * per_um
        seeds[close] += 0.3 * push[close]
        seeds[:, 0] %= nx
        seeds[:, 1] = np.clip(seeds[:, 1], r0, r1 - 1)
    band, dep = _voronoi_band(nx, r0, r1, seeds, math.sqrt(0.75), t_wall, t_cyto)
    lab[r0:r1] = band
    lab[e[4]:e[5]] = CUTICLE
    _add_chloroplasts(rng, lab, dep, r0, r1, per_um, t_wall=t_wall)
    if n_hyphae:
        _add_hyphae(rng, lab, e[0], per_um, n_hyphae)
    return lab


def random_fields(ny: int, nx: int, seed: int, scale_h: float):
    """Seeded random field state (ez, hx, hy) in SI units, hx row 0 zero.
    scale_h sets the magnetic amplitude (1/eta0 gives balanced energies)."""
    rng = np.random.default_rng(seed)
    ez = rng.standard_normal((ny, nx))
    hx = rng.standard_normal((ny, nx)) * scale_h
    hy = rng.standard_normal((ny, nx)) * scale_h
    hx[0, :] = 0.0
    return ez, hx, hy
