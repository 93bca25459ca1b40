"""The debug build of the library (FDTD_DEBUG_BOUNDS), a stand-in for a
memory checker: every index of a global-memory access that is not in range
by construction is checked in the kernel (a failure sets a bit of the
handle's error word and skips the access), and every device buffer of a
handle sits between guard bands that are checked at each synchronising
call. Small and odd grids (nx not a multiple of 32, prime ny), both
kernels, several depths and code shapes, both polarisations, a batch and an
adjoint run must finish clean and match the FP64 oracle; two planted
faults, neither of which touches memory out of range, must be reported.

The cases run in a fresh process (tests/debug_build_cases.py) that loads
libfdtd_debug.so through FDTD_LIB."""
import json
import os
import subprocess
import sys

import pytest

from gpu_common import lib, need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_runs_clean_and_reports_planted_faults():
    need_gpu()
    from paper_2512_17132_gb300 import build as b
    path = b.build(debug=True)
    env = dict(os.environ, FDTD_LIB=path)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_cases.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    cases = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    bad = [c for c in cases if not c["ok"]]
    print(f"{len(cases)} cases, {len(bad)} failed")
    for c in bad:
        print(c)
    assert r.returncode == 0 and not bad and len(cases) >= 40, r.stderr[-2000:]
    planted = [c for c in cases if c["case"].startswith("planted")]
    assert len(planted) == 3 and all(c["ok"] for c in planted)


def test_release_build_refuses_the_debug_options():
    need_gpu()
    fd = lib()
    from fdtd_inputs import config_c1b
    with fd.Simulation(config_c1b(nx=64, steps=8)) as sim:
        for opt in (fd.FDTD_OPT_DEBUG_TABLE_LIMIT, fd.FDTD_OPT_DEBUG_POKE_GUARD):
            with pytest.raises(fd.FDTDError) as e:
                fd.fdtd_set_option(sim.h, opt, 1)
            assert e.value.code == fd.FDTD_EINVAL and "debug build" in str(e.value)
