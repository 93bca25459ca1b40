"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Tolerances: fields within 1e-4 relative L2 (denominator
max(||f_ref||, 1e-2 max_n ||f_ref^n||), so that the nearly empty domain after
the pulse has left is not an ill-conditioned ratio), R and T within 2e-3
absolute; the per-half-step and temporally blocked kernels must agree bit for
bit (they share every rounding step)."""
import math

import numpy as np
import pytest

from fdtd_inputs import config_c1, config_c1b
from gpu_common import OracleTrace, component_errors, field_errors, lib, need_gpu, rel_l2

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-4
RT_TOL = 2e-3


@pytest.fixture(scope="module")
def fd():
    need_gpu()
    return lib()


def _oracle_rt(spec, steps):
    from oracle import run_rt
    r = run_rt(spec, steps)
    return r["R"], r["T"]


@pytest.fixture(scope="module")
def ref_c1():
    spec = config_c1()
    tr = OracleTrace(spec, {1500, 4000})
    from oracle.fdtd_tmz import empty_twin
    tw = empty_twin(spec).run(4000)
    p_up, p_down = tr.sim.fluxes()
    p_inc = tw.fluxes()[1] * spec.nx
    return spec, tr, (p_up / p_inc, p_down / p_inc)


@pytest.fixture(scope="module")
def ref_c1b():
    spec = config_c1b()
    tr = OracleTrace(spec, {1500, 4000})
    from oracle.fdtd_tmz import empty_twin
    tw = empty_twin(spec).run(4000)
    p_up, p_down = tr.sim.fluxes()
    p_inc = tw.fluxes()[1] * spec.nx
    return spec, tr, (p_up / p_inc, p_down / p_inc)


KERNELS = [(1, None), (2, 8), (2, 5), (2, 3)]


def _run_and_compare(fd, spec, tr, rt, kernel, K, seg=None):
    with fd.Simulation(spec, kernel=kernel, block_steps=K, seg_rows=seg) as sim:
        sim.run(1500)
        f1500 = sim.fields()
        sim.run(2500)
        f4000 = sim.fields()
        R, T = sim.flux()
        st = sim.stats()
    assert st["kernel"] == kernel
    e1 = field_errors(f1500, tr.snaps[1500], tr.max_norm)
    e2 = field_errors(f4000, tr.snaps[4000], tr.max_norm)
    c1 = component_errors(f1500, tr.snaps[1500], tr.max_norm)
    c2 = component_errors(f4000, tr.snaps[4000], tr.max_norm)
    print(f"{spec.name} kernel={kernel} K={K}: err1500={e1} err4000={e2} "
          f"(Ez, Hx, Hy alone: {c1} / {c2}) "
          f"R={R:.7f}/{rt[0]:.7f} T={T:.7f}/{rt[1]:.7f}")
    assert max(e1) < FIELD_TOL and max(e2) < FIELD_TOL
    assert abs(R - rt[0]) < RT_TOL and abs(T - rt[1]) < RT_TOL
    assert abs(R - rt[0]) < 1e-4 and abs(T - rt[1]) < 1e-4      # FP32 reaches far below


@pytest.mark.parametrize("kernel,K", KERNELS)
def test_config1_fields_and_rt(fd, ref_c1, kernel, K):
    spec, tr, rt = ref_c1
    _run_and_compare(fd, spec, tr, rt, kernel, K)


@pytest.mark.parametrize("kernel,K", KERNELS)
def test_config1b_fields_and_rt(fd, ref_c1b, kernel, K):
    spec, tr, rt = ref_c1b
    _run_and_compare(fd, spec, tr, rt, kernel, K)


@pytest.mark.parametrize("K,seg,variant", [(8, None, 1), (8, None, 0), (8, 25, 1), (7, 40, 0),
                                           (7, 40, 1), (5, 23, 1), (4, 31, 0), (2, 19, 1),
                                           (1, 17, 1), (6, 200, 0), (6, 33, 1), (3, 29, 1),
                                           (8, None, 2), (8, 27, 2), (7, 41, 2), (5, 19, 2),
                                           (3, 22, 2), (1, 18, 2), (8, None, 3), (7, None, 3),
                                           (7, 41, 3), (6, 33, 3), (4, 31, 3), (1, 18, 3),
                                           (8, None, 5), (8, 27, 5), (7, 41, 5), (6, 33, 5),
                                           (5, 19, 5), (3, 22, 5), (2, 19, 5), (1, 18, 5)])
def test_blocked_is_bitwise_equal_to_naive(fd, K, seg, variant):
    spec = config_c1b(steps=411)
    with fd.Simulation(spec, kernel=1) as a:
        a.run(411)
        fa, da = a.fields(), a.dft()
    with fd.Simulation(spec, kernel=2, block_steps=K, seg_rows=seg) as b:
        fd.fdtd_set_option(b.h, fd.FDTD_OPT_VARIANT, variant)
        b.run(200)
        b.run(211)
        fb, db = b.fields(), b.dft()
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)
    assert np.array_equal(da, db)


def test_pair_shape_is_the_default_only_where_the_labels_fit(fd):
    # code shape 5 needs S polarisation and at most 16 labels
    spec = config_c1b(steps=8)
    with fd.Simulation(spec, kernel=2) as a:
        a.run(8)
        assert a.stats()["variant"] == 5
        with pytest.raises(fd.FDTDError):
            fd.fdtd_set_option(a.h, fd.FDTD_OPT_VARIANT, 4)
    mats = np.vstack([spec.materials, np.tile([[1.3, 0.0]], (14, 1))])   # 18 labels
    lab = spec.labels.copy()
    lab[100, 7] = 17
    wide = spec.with_(materials=mats, labels=lab)
    with fd.Simulation(wide, kernel=2) as b:
        with pytest.raises(fd.FDTDError):
            fd.fdtd_set_option(b.h, fd.FDTD_OPT_VARIANT, 5)
        b.run(8)
        assert b.stats()["variant"] == 2


@pytest.mark.parametrize("nx,kernel", [(100, 2), (104, 2), (8, 2), (4, 2), (37, 1), (3, 1),
                                       (1, 1), (252, 2)])
def test_ragged_and_tiny_widths(fd, nx, kernel):
    base = config_c1b(steps=700)
    reps = -(-nx // 256)
    lab = np.tile(base.labels, (1, reps))[:, :nx].copy()
    spec = base.with_(nx=nx, labels=lab)
    tr = OracleTrace(spec, {700})
    with fd.Simulation(spec, kernel=kernel, block_steps=8, seg_rows=29) as sim:
        sim.run(700)
        f = sim.fields()
    e = field_errors(f, tr.snaps[700], tr.max_norm)
    assert max(e) < FIELD_TOL, e


def test_empty_domain_single_column_matches_reference_run(fd):
    # all air, one column: the leaf run and the internal empty-domain run
    # execute the same FP32 recurrence, so T is exactly 1 and R is leakage only
    base = config_c1(nx=1, steps=3000)
    spec = base.with_(labels=np.zeros_like(base.labels))
    with fd.Simulation(spec, kernel=1) as s:
        s.run(3000)
        R, T = s.flux()
    assert T == 1.0 and abs(R) < 1e-10
    spec8 = config_c1(nx=8, steps=3000)
    spec8 = spec8.with_(labels=np.zeros_like(spec8.labels))
    with fd.Simulation(spec8, kernel=2) as s:
        s.run(3000)
        R, T = s.flux()
    assert T == 1.0 and abs(R) < 1e-10


def test_state_roundtrip_is_exact(fd):
    spec = config_c1b(steps=600)
    with fd.Simulation(spec, kernel=2) as s:
        s.run(300)
        buf = fd.fdtd_save_state(s.h)
        s.run(300)
        f_a, d_a = s.fields(), s.dft()
        fd.fdtd_load_state(s.h, buf)
        s.run(300)
        f_b, d_b = s.fields(), s.dft()
    for x, y in zip(f_a, f_b):
        assert np.array_equal(x, y)
    assert np.array_equal(d_a, d_b)


def test_set_get_fields_roundtrip(fd):
    from fdtd_inputs import random_fields
    spec = config_c1b(steps=1).with_(source_kind=2)
    ez, hx, hy = random_fields(spec.ny, spec.nx, 5, 1.0 / 376.73)
    with fd.Simulation(spec) as s:
        s.set_fields(ez, hx, hy)
        g = s.fields()
    for a, b in zip((ez, hx, hy), g):
        assert rel_l2(b, a.astype(np.float32)) < 1e-6


def test_device_side_validation(fd):
    spec = config_c1b(steps=1)
    bad = spec.labels.copy()
    bad[100, 7] = 9
    with pytest.raises(fd.FDTDError) as e:
        fd.Simulation(spec, labels=bad)
    assert e.value.code == fd.FDTD_EINVAL and "label" in str(e.value)
    bad = spec.labels.copy()
    bad[spec.tfsf_row, 3] = 1
    with pytest.raises(fd.FDTDError) as e:
        fd.Simulation(spec, labels=bad)
    assert "air" in str(e.value)


def test_watchdog_reports_non_finite_fields(fd):
    spec = config_c1b(steps=1)
    with fd.Simulation(spec) as s:
        fd.fdtd_set_option(s.h, fd.FDTD_OPT_WATCHDOG, 16)
        ez = np.zeros((spec.ny, spec.nx), np.float32)
        ez[120, 50] = np.inf
        s.set_fields(ez)
        s.run(40)
        with pytest.raises(fd.FDTDError) as e:
            fd.fdtd_synchronize(s.h)
        assert e.value.code == fd.FDTD_EUNSTABLE


# ---------------------------------------------------------------------------
# Full-size parity on sampled outputs (light cone): after M steps from a
# random state, a cell depends only on cells within M rows/columns. The
# oracle advances a crop that holds the whole cone (plus a CPML depth where
# the crop edge is not a true domain edge) and the sampled cells must match.
# ---------------------------------------------------------------------------

def _crop_check(fd, spec, fields0, gpu_fields, samples, M):
    from oracle import TMzOracle
    ny, nx, P = spec.ny, spec.nx, spec.pml_cells
    worst = 0.0
    scale = [float(np.abs(f).max()) for f in fields0]
    for (j, i) in samples:
        m = M + 3
        top = 0 if j - m - P - 2 <= 0 else j - m - P - 2
        bot = ny if j + m + P + 2 >= ny else j + m + P + 2
        cols = np.arange(i - m - 2, i + m + 3) % nx
        sub = spec.with_(ny=bot - top, nx=len(cols),
                         labels=np.ascontiguousarray(spec.labels[top:bot][:, cols]),
                         tfsf_row=2, r_row=1, t_row=bot - top - P - 3, pml_cells=P,
                         source_kind=2)
        # keep the CPML only where the crop edge is the true domain edge
        o = TMzOracle(sub)
        if top != 0:
            o.pml_e = [blk for blk in o.pml_e if blk[0][0] != 0]
            o.pml_h = [blk for blk in o.pml_h if blk[0][0] != 1]
        if bot != ny:
            o.pml_e = [blk for blk in o.pml_e if blk[0][-1] != sub.ny - 1]
            o.pml_h = [blk for blk in o.pml_h if blk[0][-1] != sub.ny - 1]
        o.set_fields(*[np.asarray(f[top:bot][:, cols], np.float64) for f in fields0])
        if top != 0:
            o.hx[0] = fields0[1][top, cols]       # the crop's top edge is interior
        o.run(M)
        jj, ii = j - top, m + 2
        for q, (g, r) in enumerate(zip(gpu_fields, o.fields())):
            err = abs(float(g[j, i]) - r[jj, ii]) / scale[q]
            worst = max(worst, err)
    return worst


def _light_cone(fd, spec, M, n_random=24, seed=0):
    from fdtd_inputs import random_fields
    spec = spec.with_(source_kind=2)
    ez, hx, hy = random_fields(spec.ny, spec.nx, seed, 1.0 / 376.73)
    ez, hx, hy = ez.astype(np.float32), hx.astype(np.float32), hy.astype(np.float32)
    with fd.Simulation(spec, kernel=2) as s:
        s.set_fields(ez, hx, hy)
        s.run(M)
        g = s.fields()
        st = s.stats()
    rng = np.random.default_rng(seed + 1)
    ny, nx = spec.ny, spec.nx
    w = 128 - 2 * ((st["block_steps"] + 3) // 4 * 4)
    samples = [(2, 0), (9, nx - 1), (15, 1), (16, w), (ny - 1, w - 1), (ny - 9, 0),
               (ny - 16, nx - 2), (ny - 17, 3), (spec.r_row, 5), (spec.t_row + 1, w + 1),
               (st["seg_rows"], 2 * w), (st["seg_rows"] - 1, 2 * w - 1)]
    samples += [(int(rng.integers(0, ny)), int(rng.integers(0, nx))) for _ in range(n_random)]
    worst = _crop_check(fd, spec, (ez, hx, hy), g, samples, M)
    print(f"{spec.name}: light-cone worst relative error {worst:.3e} over {len(samples)} cells")
    assert worst < 2e-5


def test_light_cone_parity_config2_full_size(fd):
    from fdtd_inputs import config_c2
    _light_cone(fd, config_c2(), M=16)


def test_light_cone_parity_config3_full_size(fd):
    from fdtd_inputs import config_c3
    _light_cone(fd, config_c3(diseased=True), M=16, n_random=8)
