"""Batched runs (many simulations per launch, CUDA-graph chunks) and the
launch-shape autotuner: results must equal each simulation run alone, bit
for bit, and tuning must leave the state untouched."""
import numpy as np
import pytest

from fdtd_inputs import config_c1, config_c1b, config_c2, crop_layout
from gpu_common import lib, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    need_gpu()
    return lib()


def _specs():
    c2 = config_c2()
    return [
        config_c1b(steps=1),
        config_c1(nx=128, steps=1).with_(lambda0=700e-9),
        crop_layout(c2, ny=1500).with_(lambda0=450e-9),
        crop_layout(c2.with_(labels=np.ascontiguousarray(c2.labels[:, :1000]), nx=1000),
                    ny=2100).with_(lambda0=1450e-9),
        config_c1b(nx=100, steps=1).with_(lambda0=620e-9),
    ]


def _alone(fd, spec, steps_list):
    with fd.Simulation(spec, kernel=fd.KERNEL_BLOCKED) as s:
        for n in steps_list:
            s.run(n)
        return s.fields(), s.dft(), s.flux_raw()


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_runs_alone(fd, graph):
    specs = _specs()
    steps = [1000, 1371]                      # one full graph chunk, then odd counts
    ref = [_alone(fd, sp, steps) for sp in specs]
    sims = [fd.Simulation(sp, kernel=fd.KERNEL_BLOCKED) for sp in specs]
    with fd.Batch(sims, timing=True, graph=graph) as b:
        for n in steps:
            b.run(n)
        st = b.stats()
        got = [(s.fields(), s.dft(), s.flux_raw()) for s in sims]
    for s in sims:
        s.close()
    assert st["steps"] == sum(steps) and st["graph"] == graph
    for (fa, da, ra), (fb, db, rb) in zip(ref, got):
        for x, y in zip(fa, fb):
            assert np.array_equal(x, y)
        assert np.array_equal(da, db)
        np.testing.assert_array_equal(np.array(ra), np.array(rb))


def test_batch_with_handles_at_different_steps(fd):
    specs = _specs()[:3]
    ref = [_alone(fd, sp, [700 + 37 * i, 1100]) for i, sp in enumerate(specs)]
    sims = [fd.Simulation(sp, kernel=fd.KERNEL_BLOCKED) for sp in specs]
    for i, s in enumerate(sims):
        s.run(700 + 37 * i)
    with fd.Batch(sims) as b:
        b.run(1100)
        got = [(s.fields(), s.dft()) for s in sims]
    for s in sims:
        s.close()
    for (fa, da, _), (fb, db) in zip(ref, got):
        for x, y in zip(fa, fb):
            assert np.array_equal(x, y)
        assert np.array_equal(da, db)


def test_autotune_leaves_state_and_results_unchanged(fd):
    specs = _specs()[:4]
    ref = [_alone(fd, sp, [600, 900]) for sp in specs]
    sims = [fd.Simulation(sp, kernel=fd.KERNEL_BLOCKED) for sp in specs]
    for s in sims:
        s.run(600)
    with fd.Batch(sims) as b:
        b.autotune(2)
        b.run(900)
        st = b.stats()
        got = [(s.fields(), s.dft()) for s in sims]
    assert 1 <= st["block_steps"] <= 8
    for s in sims:
        s.close()
    for (fa, da, _), (fb, db) in zip(ref, got):
        for x, y in zip(fa, fb):
            assert np.array_equal(x, y)
        assert np.array_equal(da, db)
    spec = specs[2]
    with fd.Simulation(spec, kernel=fd.KERNEL_BLOCKED) as s:
        s.run(600)
        fd.fdtd_autotune(s.h, 2)
        s.run(900)
        f = s.fields()
    for x, y in zip(ref[2][0], f):
        assert np.array_equal(x, y)


def test_batch_member_matches_oracle(fd):
    from oracle import run_rt
    spec = config_c1b(nx=64, steps=2500).with_(lambda0=600e-9)
    from fdtd_inputs import leaf_materials  # noqa: F401  (materials stay c1b's)
    r = run_rt(spec, 2500)
    sims = [fd.Simulation(sp, kernel=fd.KERNEL_BLOCKED) for sp in [spec] + _specs()[:2]]
    with fd.Batch(sims) as b:
        b.run(2500)
        R, T = sims[0].flux()
    for s in sims:
        s.close()
    assert abs(R - r["R"]) < 2e-3 and abs(T - r["T"]) < 2e-3
    assert abs(R - r["R"]) < 1e-4 and abs(T - r["T"]) < 1e-4


def test_batch_rejects_bad_members(fd):
    spec = config_c1b(nx=37, steps=1)
    with fd.Simulation(spec) as a, fd.Simulation(config_c1b(steps=1)) as c:
        with pytest.raises(fd.FDTDError) as e:
            fd.fdtd_batch_create([c.h, a.h])
        assert "nx % 4" in str(e.value)
        with pytest.raises(fd.FDTDError):
            fd.fdtd_batch_create([c.h, c.h])


def test_shared_incident_tables_give_identical_runs(fd):
    # handles with the same source share one table store; a run that goes
    # past the store's plan regrows it. Interleaved handles must give the
    # bits of a handle run alone.
    from fdtd_inputs import config_c1b
    spec = config_c1b(nx=64, steps=1)
    with fd.Simulation(spec) as ref:
        ref.run(2600)
        want = ref.flux_raw()
        want_f = ref.fields()
    with fd.Simulation(spec) as a:
        a.run(300)                          # store planned for 300 steps
        with fd.Simulation(spec) as b:
            b.run(2600)                     # regrows the shared store
            np.testing.assert_array_equal(b.flux_raw(), want)
        a.run(2300)                         # continues from the regrown store
        np.testing.assert_array_equal(a.flux_raw(), want)
        for x, y in zip(a.fields(), want_f):
            assert np.array_equal(x, y)
