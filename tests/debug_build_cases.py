"""Cases run against the debug build of the library (FDTD_DEBUG_BOUNDS: in-kernel
index checks that record a failure and skip the access, guard bands around
the device buffers). Run as a script in a fresh process with FDTD_LIB set to
libfdtd_debug.so; prints one JSON line per case and exits non-zero if a case
fails. tests/test_gpu_debug_build.py drives it.

Every ordinary case must finish without an FDTD_EBOUNDS report and match the
FP64 oracle; the two planted cases must be reported: a run longer than the
table entries the checks admit (FDTD_OPT_DEBUG_TABLE_LIMIT; every access stays
inside the allocated tables) and a byte written into a guard band from the
host (FDTD_OPT_DEBUG_POKE_GUARD)."""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from fdtd_inputs import POL_P, config_c1                     # noqa: E402
from fdtd_inputs.configs import SOURCE_CW                      # noqa: E402

FIELD_TOL = 1e-4
STEPS = 300


def small_spec(nx, ny, P, seed, pol=0):
    """A small grid with its own row layout (CPML of P rows, monitors and the
    TF/SF row inside), three random labels, a CW source from step 0."""
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, 3, size=(ny, nx)).astype(np.uint8)
    lab[:P + 5] = 0
    mats = np.array([[1.0, 0.0], [1.45, 0.0], [1.42, 0.02]])
    return config_c1(nx=nx, steps=STEPS).with_(
        ny=ny, nx=nx, labels=lab, materials=mats, pml_cells=P, r_row=P + 1, tfsf_row=P + 3,
        t_row=ny - P - 3, source_kind=SOURCE_CW, polarization=pol)


def oracle(spec):
    from oracle import TMzOracle
    from oracle.fdtd_tez import TEzOracle
    o = (TEzOracle if spec.polarization else TMzOracle)(spec)
    o.run(spec.steps)
    return o.fields()


def rel_err(got, ref):
    num = math.sqrt(sum(float(np.sum((np.asarray(g, np.float64) - r) ** 2))
                        for g, r in zip(got, ref)))
    den = math.sqrt(sum(float(np.sum(np.asarray(r) ** 2)) for r in ref))
    return num / max(den, 1e-300)


def main():
    from paper_2512_17132_gb300 import fdtd
    lib_path = os.environ.get("FDTD_LIB", "")
    assert lib_path.endswith("libfdtd_debug.so"), lib_path
    fdtd.load_library()
    import torch
    torch.cuda.set_device(0)
    failures = 0

    def report(name, ok, **kw):
        nonlocal failures
        failures += 0 if ok else 1
        print(json.dumps({"case": name, "ok": bool(ok), **kw}), flush=True)

    # small and odd grids: both kernels, several depths and code shapes
    grids = [(8, 40, 4), (12, 41, 4), (36, 43, 5), (60, 64, 6), (100, 97, 8), (4, 53, 4),
             (132, 59, 6), (37, 47, 4), (3, 31, 3)]
    for g, (nx, ny, P) in enumerate(grids):
        for pol in (0, 1):
            spec = small_spec(nx, ny, P, seed=g, pol=pol)
            ref = oracle(spec)
            runs = [(1, None, None)]
            if nx % 4 == 0:
                runs += [(2, 1, 2), (2, 3, 2), (2, 8, 2)]
                if pol == 0:
                    runs += [(2, 8, 5), (2, 5, 5), (2, 8, 0)]
            for kernel, K, shape in runs:
                name = f"grid {nx}x{ny} P={P} pol={'SP'[pol]} kernel={kernel} K={K} shape={shape}"
                try:
                    with fdtd.Simulation(spec, kernel=kernel, block_steps=K) as sim:
                        if shape is not None:
                            fdtd.fdtd_set_option(sim.h, fdtd.FDTD_OPT_VARIANT, shape)
                        sim.run(STEPS // 2)
                        sim.run(STEPS - STEPS // 2)
                        sim.flux_raw()
                        err = rel_err(sim.fields(), ref)
                    report(name, err <= FIELD_TOL, err=err)
                except fdtd.FDTDError as e:
                    report(name, False, error=str(e))

    # a batch of three small grids and a small adjoint
    specs = [small_spec(nx, ny, P, seed=10 + i) for i, (nx, ny, P) in
             enumerate([(8, 40, 4), (36, 43, 5), (60, 64, 6)])]
    try:
        sims = [fdtd.Simulation(sp, kernel=2) for sp in specs]
        with fdtd.Batch(sims) as b:
            b.run(STEPS)
            errs = [rel_err(s.fields(), oracle(sp)) for s, sp in zip(sims, specs)]
        for s in sims:
            s.close()
        report("batch of three small grids", max(errs) <= FIELD_TOL, err=max(errs))
    except fdtd.FDTDError as e:
        report("batch of three small grids", False, error=str(e))
    try:
        base = small_spec(36, 64, 6, seed=20).with_(source_kind=0)
        sp = base.with_(steps=2000)
        with fdtd.Simulation(sp) as sim:
            g = sim.gradient(2000, wR=1.0, wT=0.5, every=250)
        report("adjoint 36x64", bool(np.all(np.isfinite(g["g_n"]))))
    except fdtd.FDTDError as e:
        report("adjoint 36x64", False, error=str(e))

    # planted: the checks admit 100 table entries, the run needs 300
    spec = small_spec(60, 64, 6, seed=30)
    for kernel in (1, 2):
        name = f"planted table limit, kernel={kernel}"
        try:
            with fdtd.Simulation(spec, kernel=kernel) as sim:
                fdtd.fdtd_set_option(sim.h, fdtd.FDTD_OPT_DEBUG_TABLE_LIMIT, 100)
                sim.run(STEPS)
                sim.flux_raw()
            report(name, False, error="not reported")
        except fdtd.FDTDError as e:
            report(name, e.code == fdtd.FDTD_EBOUNDS and "table entry" in str(e), error=str(e))
    # planted: one byte written into the guard band behind Ez
    name = "planted guard-band write"
    try:
        with fdtd.Simulation(spec, kernel=2) as sim:
            sim.run(16)
            sim.flux_raw()                               # clean so far
            fdtd.fdtd_set_option(sim.h, fdtd.FDTD_OPT_DEBUG_POKE_GUARD, 1)
            sim.flux_raw()
        report(name, False, error="not reported")
    except fdtd.FDTDError as e:
        report(name, e.code == fdtd.FDTD_EBOUNDS and "guard band" in str(e), error=str(e))
    return 1 if failures else 0


if __name__ == "__main__":
    sys.exit(main())
