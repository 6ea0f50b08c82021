"""Differentiable contact volumes: torch.autograd functions over the SH
coefficients of a suspension.

Forward: upsample X0 and X1 (Sec. 3.1.2), detect contacts (Alg. 1, Eq. 3.1)
and return the interference volume of every candidate vesicle pair (Eq. 3.2,
summed per pair as in Alg. 2).  Backward: the vector-Jacobian product with
respect to the end-of-step coefficients, J^T g with J = dV/dX1 (Sec. 3.2)
followed by the adjoint of the upsampling.  The forward keeps no meshes,
contact lists or gradient rows: the backward recomputes them from the saved
coefficients (the library's detection is deterministic, so it reproduces the
forward's pair list exactly, which is checked).

Every step runs in libstiv's kernels; this module only passes pointers.
The start-of-step coefficients are constants of the step (the method moves
X1 and keeps X0 fixed): their block of the returned gradient is zero.
"""
from __future__ import annotations

import dataclasses

import torch

from . import stiv as S


class StivVolumes(torch.autograd.Function):
    """V_pair = StivVolumes.apply(coef, engine, ds).

    coef: float64 device tensor in the coefficient layout of ``ds`` (per
    vesicle [2 time][3 coord][(p+1)^2] at ds.coef_off).  engine: a
    ``stiv.Stiv`` handle; ds: a ``stiv.DeviceScene`` giving orders, offsets
    and the vertex buffer (its own ``coef`` is not read).  Returns the volume
    of each candidate vesicle pair (i < j, periodic shift), in the library's
    pair order."""

    @staticmethod
    def forward(ctx, coef, engine, ds):
        if coef.dtype != torch.float64 or not coef.is_cuda:
            raise TypeError("coef must be a float64 CUDA tensor")
        if coef.numel() != ds.coef.numel():
            raise ValueError("coef does not match the scene's coefficient layout")
        dsc = dataclasses.replace(ds, coef=coef.detach().contiguous())
        r = engine.step(dsc, grad=False)
        V = r["V_pair"].clone()
        ctx.engine, ctx.ds = engine, dsc
        ctx.npairs = int(r["counts"][S.C_PAIRS])
        ctx.pairs = (r["i"].clone(), r["j"].clone(), r["shift"].clone())
        return V

    @staticmethod
    def backward(ctx, gV):
        eng, ds = ctx.engine, ctx.ds
        r = eng.step(ds, grad=True)
        if int(r["counts"][S.C_PAIRS]) != ctx.npairs or not all(
                torch.equal(a, b) for a, b in zip((r["i"], r["j"], r["shift"]), ctx.pairs)):
            raise RuntimeError("recomputed candidate pairs differ from the forward pass")
        st = torch.cuda.current_stream().cuda_stream
        b = eng.buf
        w = gV.detach().to(torch.float64).contiguous()
        gX = torch.zeros(ds.verts.numel(), dtype=torch.float64, device=ds.coef.device)
        S.stiv_grad_scatter(eng.h, st, ds.p.data_ptr(), b.contacts_struct(), b.counts.data_ptr(), w.data_ptr(),
                            b.grad.data_ptr(), b.gves.data_ptr(), b.gvid.data_ptr(), ds.vert_off.data_ptr(),
                            gX.data_ptr())
        gcoef = torch.empty_like(ds.coef)
        S.stiv_grad_to_coef(eng.h, st, ds.n, ds.p_max, ds.p.data_ptr(), ds.coef_off.data_ptr(),
                            ds.vert_off.data_ptr(), gX.data_ptr(), gcoef.data_ptr())
        return gcoef, None, None


def stiv_volumes(coef: torch.Tensor, engine: "S.Stiv", ds: "S.DeviceScene") -> torch.Tensor:
    """Per-pair interference volumes, differentiable with respect to coef."""
    return StivVolumes.apply(coef, engine, ds)


def stiv_sum(coef: torch.Tensor, engine: "S.Stiv", ds: "S.DeviceScene") -> torch.Tensor:
    """Total interference volume of the step (sum over vesicle pairs)."""
    return StivVolumes.apply(coef, engine, ds).sum()
