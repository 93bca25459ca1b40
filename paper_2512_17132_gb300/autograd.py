"""torch.autograd functions over the CUDA discrete adjoint.

FDTDMapFunction:   (eps_r map, sigma map) -> (R, T); gradients per cell.
FDTDTableFunction: (n, kappa) per label     -> (R, T); gradients per label.

The forward runs fdtd_forward_checkpointed on a fresh handle; backward calls
fdtd_backward with (wR, wT) = the incoming gradients of (R, T), which is the
vector-Jacobian product because J = wR R + wT T is linear in (wR, wT). All
arithmetic runs in libfdtd.so; torch only carries tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fdtd


class FDTDMapFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_r, sigma, spec, steps, every):
        e = eps_r.detach().to(torch.float64).contiguous()
        s = sigma.detach().to(torch.float64).contiguous()
        sim = fdtd.Simulation(spec, eps_r=e, sigma=s)
        fdtd.fdtd_forward_checkpointed(sim.h, steps, every)
        R, T = sim.flux()
        ctx.sim = sim
        ctx.meta = (spec.ny, spec.nx, eps_r.device, eps_r.dtype)
        return torch.tensor([R, T], dtype=torch.float64, device=eps_r.device)

    @staticmethod
    def backward(ctx, grad_rt):
        ny, nx, dev, dt = ctx.meta
        wR, wT = (float(v) for v in grad_rt.detach().cpu().tolist())
        res = fdtd.fdtd_backward(ctx.sim.h, wR, wT, ny, nx)
        ctx.sim.close()
        ge = torch.from_numpy(res["g_eps"]).to(device=dev, dtype=dt)
        gs = torch.from_numpy(res["g_sigma"]).to(device=dev, dtype=dt)
        return ge, gs, None, None, None


class FDTDTableFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, table, spec, steps, every):
        mats = table.detach().cpu().to(torch.float64).numpy()
        sp = spec.with_(materials=np.ascontiguousarray(mats))
        sim = fdtd.Simulation(sp)
        fdtd.fdtd_forward_checkpointed(sim.h, steps, every)
        R, T = sim.flux()
        ctx.sim = sim
        ctx.meta = (sp.ny, sp.nx, len(mats), table.device, table.dtype)
        return torch.tensor([R, T], dtype=torch.float64, device=table.device)

    @staticmethod
    def backward(ctx, grad_rt):
        ny, nx, nl, dev, dt = ctx.meta
        wR, wT = (float(v) for v in grad_rt.detach().cpu().tolist())
        res = fdtd.fdtd_backward(ctx.sim.h, wR, wT, ny, nx, nl)
        ctx.sim.close()
        g = np.stack([res["g_n"], res["g_k"]], axis=1)
        return torch.from_numpy(g).to(device=dev, dtype=dt), None, None, None


def reflectance_transmittance(eps_r, sigma, spec, steps, every=500):
    """(R, T) as a differentiable function of per-cell eps_r and sigma."""
    return FDTDMapFunction.apply(eps_r, sigma, spec, steps, every)


def reflectance_transmittance_table(table, spec, steps, every=500):
    """(R, T) as a differentiable function of the (n, kappa) label table."""
    return FDTDTableFunction.apply(table, spec, steps, every)
