"""Argument checks of the allocation-free entry point's Python binding, on
the CPU: tensors of the wrong type, layout, size or device are rejected
before the library is called, so none of them can reach a kernel."""
import numpy as np
import pytest
import torch

from fdtd_inputs import config_c1b
from paper_2512_17132_gb300 import fdtd


def _args(ny=256, nx=256, P=16):
    f = [torch.zeros(ny * nx, dtype=torch.float32) for _ in range(3)]
    f += [torch.zeros(2 * P * nx, dtype=torch.float32) for _ in range(2)]
    o = [torch.zeros_like(x) for x in f]
    lab = torch.zeros(ny * nx, dtype=torch.uint8)
    return lab, f, o


def _call(lab, f, o):
    spec = config_c1b(steps=8)
    fdtd.fdtd_blocked_advance_noalloc(fdtd.make_grid(spec), lab, spec.materials,
                                      spec.lambda0, f, o, 8)


def _rejects(lab, f, o, word):
    with pytest.raises(fdtd.FDTDError) as e:
        _call(lab, f, o)
    assert e.value.code == fdtd.FDTD_EINVAL and word in str(e.value)


def test_wrong_dtypes_are_rejected():
    lab, f, o = _args()
    _rejects(lab.to(torch.int32), f, o, "uint8")
    f2 = list(f)
    f2[1] = f2[1].double()
    _rejects(lab, f2, o, "float32")
    o2 = list(o)
    o2[3] = o2[3].half()
    _rejects(lab, f, o2, "float32")


def test_short_or_strided_buffers_are_rejected():
    lab, f, o = _args()
    _rejects(lab[:-1], f, o, "elements")
    f2 = list(f)
    f2[0] = f2[0][:1000]
    _rejects(lab, f2, o, "elements")
    o2 = list(o)
    o2[4] = torch.zeros(2 * 2 * 16 * 256, dtype=torch.float32)[::2]
    _rejects(lab, f, o2, "contiguous")
    _rejects(lab, f[:4], o, "five")


def test_host_tensors_are_rejected_before_any_launch():
    lab, f, o = _args()
    _rejects(lab, f, o, "CUDA device")
