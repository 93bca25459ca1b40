"""P polarisation (TEz) through the C ABI against the FP64 TEz oracle.

Same bars as the S path: fields within 1e-4 relative L2 (centre field Hz;
edge vector (Ex, Ey)), R and T within 2e-3 absolute (and 1e-4 in practice),
bit-for-bit equality of the per-half-step and the temporally blocked
kernels, and bit-for-bit equality of the P and S runs of an all-air domain
(the TEz/TMz duality holds exactly on the lattice and in FP32)."""
import numpy as np
import pytest

from fdtd_inputs import POL_P, POL_S, config_c1b
from gpu_common import OracleTrace, field_errors, lib, need_gpu

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-4
RT_TOL = 2e-3


@pytest.fixture(scope="module")
def fd():
    need_gpu()
    return lib()


@pytest.fixture(scope="module")
def ref_c1b_p():
    from oracle.fdtd_tez import empty_twin_tez
    spec = config_c1b().with_(polarization=POL_P)
    tr = OracleTrace(spec, {1500, 4000})
    tw = empty_twin_tez(spec).run(4000)
    p_up, p_down = tr.sim.fluxes()
    p_inc = tw.fluxes()[1] * spec.nx
    return spec, tr, (p_up / p_inc, p_down / p_inc)


@pytest.mark.parametrize("kernel,K", [(1, None), (2, 8), (2, 5), (2, 3)])
def test_config1b_p_fields_and_rt(fd, ref_c1b_p, kernel, K):
    spec, tr, rt = ref_c1b_p
    with fd.Simulation(spec, kernel=kernel, block_steps=K) as sim:
        sim.run(1500)
        f1500 = sim.fields()
        sim.run(2500)
        f4000 = sim.fields()
        R, T = sim.flux()
        st = sim.stats()
    assert st["kernel"] == kernel
    e1 = field_errors(f1500, tr.snaps[1500], tr.max_norm)
    e2 = field_errors(f4000, tr.snaps[4000], tr.max_norm)
    print(f"c1b P kernel={kernel} K={K}: err1500={e1} err4000={e2} "
          f"R={R:.7f}/{rt[0]:.7f} T={T:.7f}/{rt[1]:.7f}")
    assert max(e1) < FIELD_TOL and max(e2) < FIELD_TOL
    assert abs(R - rt[0]) < RT_TOL and abs(T - rt[1]) < RT_TOL
    assert abs(R - rt[0]) < 1e-4 and abs(T - rt[1]) < 1e-4


@pytest.mark.parametrize("variant", [2, 3, 5])
@pytest.mark.parametrize("K,seg", [(8, None), (8, 27), (7, 41), (5, 19), (3, 22), (1, 18)])
def test_p_blocked_is_bitwise_equal_to_naive(fd, K, seg, variant):
    spec = config_c1b(steps=411).with_(polarization=POL_P)
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


@pytest.mark.parametrize("kernel", [1, 2])
def test_all_air_p_state_equals_s_state(fd, kernel):
    # in air the P run in (eta0 Hz, -Ex, -Ey) is the S run in (Ez, eta0 Hx,
    # eta0 Hy), rounding step by rounding step
    base = config_c1b(steps=900)
    spec = base.with_(labels=np.zeros_like(base.labels))
    with fd.Simulation(spec, kernel=kernel) as s, \
            fd.Simulation(spec.with_(polarization=POL_P), kernel=kernel) as p:
        s.run(900)
        p.run(900)
        assert bytes(fd.fdtd_save_state(s.h)) == bytes(fd.fdtd_save_state(p.h))
        assert s.flux() == p.flux()
        fs, fp = s.fields(), p.fields()
    assert np.abs(fs[0]).max() > 0.1
    np.testing.assert_allclose(fp[0] * 376.730313412, fs[0], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(-fp[1], fs[1] * 376.730313412, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("nx,kernel", [(100, 2), (8, 2), (4, 2), (37, 1), (3, 1), (1, 1)])
def test_p_ragged_and_tiny_widths(fd, nx, kernel):
    base = config_c1b(steps=700)
    reps = -(-nx // 256)
    lab = np.tile(base.labels, (1, reps))[:, :nx].copy()
    spec = base.with_(nx=nx, labels=lab, polarization=POL_P)
    tr = OracleTrace(spec, {700})
    with fd.Simulation(spec, kernel=kernel, block_steps=8, seg_rows=29) as sim:
        sim.run(700)
        f = sim.fields()
    e = field_errors(f, tr.snaps[700], tr.max_norm)
    assert max(e) < FIELD_TOL, e


def test_p_set_get_fields_and_dft_units(fd):
    # the exchanged fields are SI (Hz in A/m, Ex and Ey in V/m)
    from oracle.fdtd_tez import TEzOracle
    spec = config_c1b(steps=300).with_(polarization=POL_P)
    rng = np.random.default_rng(3)
    hz = (rng.standard_normal((spec.ny, spec.nx)) / 376.73).astype(np.float32)
    ex = rng.standard_normal((spec.ny, spec.nx)).astype(np.float32)
    ey = rng.standard_normal((spec.ny, spec.nx)).astype(np.float32)
    ex[0] = 0.0
    o = TEzOracle(spec)
    o.hz, o.ex, o.ey = hz.astype(np.float64), ex.astype(np.float64), ey.astype(np.float64)
    o.run(300)
    with fd.Simulation(spec, kernel=2) as sim:
        sim.set_fields(hz, ex, ey)
        back = sim.fields()
        for x, y in zip(back, (hz, ex, ey)):
            np.testing.assert_allclose(x, y, rtol=2e-7, atol=1e-12)
        sim.run(300)
        f = sim.fields()
        d = sim.dft()
    err = field_errors(f, o.fields(), [np.linalg.norm(o.hz), np.linalg.norm(o.ex)])
    assert max(err) < FIELD_TOL, err
    ref = np.stack([o.dft["h_r"], o.dft["e_r"], o.dft["h_t"], o.dft["e_t"]])
    assert np.abs(d - ref).max() <= 1e-4 * np.abs(ref).max()


def test_p_batch_matches_single_runs(fd):
    specs = [config_c1b(nx=128, steps=600, seed=s).with_(polarization=POL_P) for s in (1, 2, 3)]
    single = []
    for sp in specs:
        with fd.Simulation(sp) as s:
            s.run(600)
            single.append(s.flux_raw())
    sims = [fd.Simulation(sp) for sp in specs]
    try:
        with fd.Batch(sims) as b:
            b.run(600)
        for s, ref in zip(sims, single):
            np.testing.assert_array_equal(s.flux_raw(), ref)
    finally:
        for s in sims:
            s.close()


def test_unpolarized_sweep_matches_oracle(fd):
    from oracle import run_rt
    from oracle.fdtd_tez import run_rt_tez, unpolarized
    from paper_2512_17132_gb300.campaign import run_unpolarized
    spec = config_c1b(nx=64, steps=3000)
    got = run_unpolarized([spec], autotune=False)
    ref = unpolarized(run_rt(spec), run_rt_tez(spec))
    assert abs(got["R"][0] - ref["R"]) < 1e-4 and abs(got["T"][0] - ref["T"]) < 1e-4
    assert got["R_s"][0] != got["R_p"][0]


def test_p_validation_errors(fd):
    spec = config_c1b(steps=10).with_(polarization=POL_P)
    with pytest.raises(fd.FDTDError) as e:
        fd.Simulation(spec.with_(materials=np.tile(spec.materials, (5, 1))))   # 20 labels
    assert e.value.code == fd.FDTD_EINVAL
    eps = np.ones((spec.ny, spec.nx))
    with pytest.raises(fd.FDTDError):
        fd.Simulation(spec, eps_r=eps, sigma=np.zeros_like(eps))
    with pytest.raises(fd.FDTDError):
        fd.Simulation(spec.with_(polarization=2))
    with fd.Simulation(spec) as p:
        with pytest.raises(fd.FDTDError) as e:
            fd.fdtd_forward_checkpointed(p.h, 10, 5)
        assert e.value.code == fd.FDTD_EINVAL
        with fd.Simulation(spec.with_(polarization=POL_S)) as s:
            with pytest.raises(fd.FDTDError):
                fd.Batch([s, p])


# Full-size parity on sampled outputs: after M steps from a random state a
# cell depends only on cells within M rows/columns, so the TEz oracle
# advances a crop holding the light cone.

def _crop_check_p(spec, fields0, gpu_fields, samples, M):
    from oracle.fdtd_tez import TEzOracle
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
        o = TEzOracle(sub)
        if top != 0:                  # the crop's top is interior: no CPML there
            o.pml_c = [blk for blk in o.pml_c if blk[0][0] != 0]
            o.pml_x = [blk for blk in o.pml_x if blk[0][0] != 1]
        if bot != ny:
            o.pml_c = [blk for blk in o.pml_c if blk[0][-1] != sub.ny - 1]
            o.pml_x = [blk for blk in o.pml_x if blk[0][-1] != sub.ny - 1]
        # where the crop's top is interior, its edge row 0 stays frozen in the
        # oracle; the light cone of the sample never reaches it
        o.hz, o.ex, o.ey = [np.asarray(f[top:bot][:, cols], np.float64) for f in fields0]
        o.run(M)
        jj, ii = j - top, m + 2
        for q, (g, r) in enumerate(zip(gpu_fields, o.fields())):
            worst = max(worst, abs(float(g[j, i]) - r[jj, ii]) / scale[q])
    return worst


def test_light_cone_parity_config2_full_size_p(fd):
    from fdtd_inputs import config_c2
    spec = config_c2().with_(source_kind=2, polarization=POL_P)
    M = 16
    rng = np.random.default_rng(5)
    hz = (rng.standard_normal((spec.ny, spec.nx)) / 376.73).astype(np.float32)
    ex = rng.standard_normal((spec.ny, spec.nx)).astype(np.float32)
    ey = rng.standard_normal((spec.ny, spec.nx)).astype(np.float32)
    ex[0] = 0.0
    with fd.Simulation(spec, kernel=2) as s:
        s.set_fields(hz, ex, ey)
        s.run(M)
        g = s.fields()
        st = s.stats()
    ny, nx = spec.ny, spec.nx
    w = 128 - 2 * ((st["block_steps"] + 3) // 4 * 4)
    samples = [(2, 0), (9, nx - 1), (15, 1), (16, w), (ny - 1, w - 1), (ny - 9, 0),
               (ny - 16, nx - 2), (ny - 17, 3), (st["seg_rows"], 2 * w),
               (st["seg_rows"] - 1, 2 * w - 1)]
    samples += [(int(rng.integers(0, ny)), int(rng.integers(0, nx))) for _ in range(16)]
    worst = _crop_check_p(spec, (hz, ex, ey), g, samples, M)
    print(f"c2 P: light-cone worst relative error {worst:.3e} over {len(samples)} cells")
    assert worst < 2e-5
