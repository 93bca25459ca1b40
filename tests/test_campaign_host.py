"""Host logic of the spectrum/slice campaign (no GPU): slicing along x,
the bookkeeping of run_campaign, the slice and polarisation averages, and
the grouping of run_sweep into one-polarisation batches."""
import numpy as np
import pytest

from fdtd_inputs import POL_P, POL_S, config_c1b
from paper_2512_17132_gb300 import campaign


def test_slices_partition_the_cross_section():
    spec = config_c1b(nx=203, steps=10)
    cut = campaign.slice_specs(spec, 5)
    widths = [w for _, w in cut]
    assert widths == [40, 40, 40, 40, 43] and sum(widths) == 203
    assert all(sp.nx == w for sp, w in cut)
    assert np.array_equal(np.concatenate([sp.labels for sp, _ in cut], axis=1), spec.labels)
    assert all(sp.nx % 4 == 0 for sp, _ in cut[:-1])
    with pytest.raises(ValueError):
        campaign.slice_specs(spec.with_(nx=12, labels=spec.labels[:, :12]), 5)


def test_campaign_bookkeeping_and_averages():
    seen = []

    def fake_runner(specs, steps):
        seen.extend(specs)
        R = np.array([s.lambda0 * 1e6 + 0.01 * s.nx + 0.5 * s.polarization for s in specs])
        return R, 1.0 - 2.0 * R

    make = lambda lam: config_c1b(nx=100, steps=7).with_(lambda0=lam)
    out = campaign.run_campaign(make, [500e-9, 700e-9], n_slices=3, runner=fake_runner)
    assert len(seen) == 2 * 3 * 2
    assert out["R_runs"].shape == (2, 3, 2)
    assert list(out["widths"]) == [32.0, 32.0, 36.0]
    for l, lam in enumerate((500e-9, 700e-9)):
        for s, w in enumerate((32, 32, 36)):
            for p, pol in enumerate((POL_S, POL_P)):
                assert out["R_runs"][l, s, p] == pytest.approx(lam * 1e6 + 0.01 * w + 0.5 * pol)
    wk = np.array([32, 32, 36]) / 100.0
    np.testing.assert_allclose(out["R_pol"], np.einsum("lsp,s->lp", out["R_runs"], wk))
    np.testing.assert_allclose(out["R"], out["R_pol"].mean(axis=1))
    np.testing.assert_allclose(out["A"], 1.0 - out["R"] - out["T"])
    # width-weighted = the plain mean of the slices when the widths are equal
    out2 = campaign.run_campaign(make, [500e-9], n_slices=5, runner=fake_runner)
    assert out2["R_pol"][0, 0] == pytest.approx(out2["R_runs"][0, :, 0].mean())


def test_run_sweep_batches_one_polarisation_at_a_time(monkeypatch):
    batches = []

    class FakeSim:
        def __init__(self, spec):
            self.spec = spec

        def flux(self):
            return self.spec.lambda0, float(self.spec.polarization)

        def run(self, n):
            self.spec = self.spec.with_(lambda0=self.spec.lambda0)

        def close(self):
            pass

        def __enter__(self):
            return self

        def __exit__(self, *a):
            pass

    class FakeBatch:
        def __init__(self, sims):
            pols = {s.spec.polarization for s in sims}
            assert len(pols) == 1
            batches.append((pols.pop(), len(sims)))

        def autotune(self, n):
            pass

        def run(self, n):
            pass

        def __enter__(self):
            return self

        def __exit__(self, *a):
            pass

    monkeypatch.setattr(campaign.fdtd, "Simulation", FakeSim)
    monkeypatch.setattr(campaign.fdtd, "Batch", FakeBatch)
    base = config_c1b(nx=64, steps=5)
    specs = [base.with_(lambda0=(400 + i) * 1e-9, polarization=i % 2) for i in range(7)]
    specs.append(base.with_(nx=7, labels=base.labels[:, :7], lambda0=999e-9))
    R, T = campaign.run_sweep(specs, chunk=2)
    assert sorted(batches) == [(0, 2), (0, 2), (1, 1), (1, 2)]
    np.testing.assert_allclose(R, [s.lambda0 for s in specs])
    np.testing.assert_allclose(T, [float(s.polarization) for s in specs])
