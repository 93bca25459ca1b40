"""The C-ABI library builds, loads without a GPU and exports every function
include/*.h declares; argument validation that needs no device runs here."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from conftest import ROOT

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def lib():
    from paper_2512_17132_gb300 import build as b
    b.build()
    from paper_2512_17132_gb300 import fdtd
    return fdtd.load_library()


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fdtd_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_problem_statement_calls():
    names = declared_functions()
    for must in ("fdtd_create", "fdtd_run", "fdtd_flux", "fdtd_destroy", "fdtd_get_fields",
                 "fdtd_save_state", "fdtd_load_state", "fdtd_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_wraps_every_declared_symbol():
    from paper_2512_17132_gb300 import fdtd
    for n in declared_functions():
        assert callable(getattr(fdtd, n, None)), n


def _spec():
    from fdtd_inputs import config_c1
    return config_c1(nx=8, steps=10)


def _create_code(lib, spec, **over):
    from paper_2512_17132_gb300 import fdtd
    g = fdtd.make_grid(spec)
    for k, v in over.items():
        setattr(g, k, v)
    src = fdtd.make_source(spec)
    lab = np.ascontiguousarray(spec.labels)
    mats = (fdtd.fdtd_material * len(spec.materials))(
        *[fdtd.fdtd_material(float(n), float(k)) for n, k in spec.materials])
    out = ctypes.c_void_p()
    code = lib.fdtd_create(ctypes.byref(g), lab.ctypes.data_as(ctypes.c_void_p), mats,
                           len(spec.materials), ctypes.byref(src), None, ctypes.byref(out))
    return code, out, lib.fdtd_last_error(None).decode()


@pytest.mark.parametrize("field,value,needle", [
    ("dt", 0.75 * 20e-9 / 299792458.0, "CFL"),
    ("r_row", 30, "r_row"),
    ("t_row", 250, "t_row"),
    ("pml_kappa_max", 0.5, "CPML"),
    ("nx", 0, "nx"),
])
def test_invalid_grid_is_rejected_before_touching_the_device(lib, field, value, needle):
    code, out, msg = _create_code(lib, _spec(), **{field: value})
    assert code == -1 and not out.value
    assert needle in msg


def test_null_arguments_are_rejected(lib):
    out = ctypes.c_void_p()
    assert lib.fdtd_create(None, None, None, 0, None, None, ctypes.byref(out)) == -1
    assert lib.fdtd_run(None, 10) == -1
    assert lib.fdtd_flux(None, None, None) == -1
    lib.fdtd_destroy(None)
