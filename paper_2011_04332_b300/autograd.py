"""PyTorch autograd for the npFEM step and for checkpointed rollouts (FP64).

The gradient of the quasi-Newton step comes from the library's hand-written reverse
mode (npfem_step_adjoint); PyTorch only carries the tensors and chains the steps.
Material weights enter as a [ntypes, 4] tensor (w_strain, w_bend, w_area, w_vol) that
must equal the materials the batch's cell types were built with: the factorised global
matrix depends on them, so new weight values need new cell types (see
`Calibration.rebuild`).

Rollouts differentiate through the library's rollout adjoint (npfem_rollout_adjoint):
it keeps a checkpoint of (x, v) every `ckpt_every` steps, recomputes each segment forward
from its checkpoint and runs the per-step adjoints in reverse, so memory grows with
nsteps/ckpt_every + ckpt_every states instead of nsteps.  The forward pass here only
steps and keeps (x0, v0).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np
import torch

from . import native


def _type_sum(batch: native.Batch, gw_cells: torch.Tensor, type_of_cell: torch.Tensor, ntypes: int):
    out = torch.zeros((ntypes, 4), dtype=torch.float64, device=gw_cells.device)
    out.index_add_(0, type_of_cell.long(), gw_cells)
    return out


class StepFunction(torch.autograd.Function):
    """(x_{n+1}, v_{n+1}) = step(x_n, v_n, f, weights) on an FP64 batch."""

    @staticmethod
    def forward(ctx, x, v, f, weights, batch, type_of_cell, iters):
        xo, vo = x.detach().clone(), v.detach().clone()
        batch.step(xo, vo, f.detach(), iters=iters)
        ctx.save_for_backward(x.detach(), v.detach(), f.detach(), type_of_cell, iters)
        ctx.batch = batch
        ctx.ntypes = weights.shape[0]
        return xo, vo

    @staticmethod
    def backward(ctx, gxn, gvn):
        x, v, f, toc, iters = ctx.saved_tensors
        b = ctx.batch
        gxn = torch.zeros_like(x) if gxn is None else gxn.contiguous()
        gvn = torch.zeros_like(x) if gvn is None else gvn.contiguous()
        gx, gv, gf = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
        gw = torch.empty((b.ncells, 4), dtype=torch.float64, device=x.device)
        b.step_adjoint(x, v, f, gxn, gvn, gx, gv, gf, gw, iters=iters)
        return gx, gv, gf, _type_sum(b, gw, toc, ctx.ntypes), None, None, None


def step(batch: native.Batch, x, v, f, weights, type_of_cell, iters):
    return StepFunction.apply(x, v, f, weights, batch, type_of_cell, iters)


class RolloutFunction(torch.autograd.Function):
    """nsteps steps with constant forces; returns (x_N, v_N)."""

    @staticmethod
    def forward(ctx, x0, v0, f, weights, batch, type_of_cell, iters, nsteps, ckpt_every):
        x, v = x0.detach().clone(), v0.detach().clone()
        for _ in range(nsteps):
            batch.step(x, v, f.detach(), iters=iters)
        ctx.save_for_backward(x0.detach(), v0.detach(), f.detach(), iters)
        ctx.batch, ctx.nsteps, ctx.ckpt_every, ctx.ntypes = batch, nsteps, ckpt_every, weights.shape[0]
        return x, v

    @staticmethod
    def backward(ctx, gxn, gvn):
        x0, v0, f, iters = ctx.saved_tensors
        b = ctx.batch
        gxn = torch.zeros_like(x0) if gxn is None else gxn.contiguous()
        gvn = None if gvn is None else gvn.contiguous()
        gx, gv, gf = torch.empty_like(x0), torch.empty_like(x0), torch.empty_like(x0)
        gw = torch.empty((ctx.ntypes, 4), dtype=torch.float64, device=x0.device)
        b.rollout_adjoint(x0, v0, f, gxn, gvn, gx, gv, gf, gw, ctx.nsteps, ctx.ckpt_every, iters=iters)
        return gx, gv, gf, gw, None, None, None, None, None


def rollout(batch: native.Batch, x0, v0, f, weights, type_of_cell, iters, nsteps: int, ckpt_every: int):
    return RolloutFunction.apply(x0, v0, f, weights, batch, type_of_cell, iters, nsteps, ckpt_every)


def end_vertex_sets(verts: np.ndarray, frac: float = 0.05):
    """Fixed index sets of the `frac` extreme vertices along the rest x and y axes."""
    n = verts.shape[0]
    k = max(1, int(round(frac * n)))
    ox = np.argsort(verts[:, 0], kind="stable")
    oy = np.argsort(verts[:, 1], kind="stable")
    return (ox[:k], ox[-k:]), (oy[:k], oy[-k:])


def diameters(x: torch.Tensor, offsets: Sequence[int], sets) -> torch.Tensor:
    """Per-cell axial and transverse diameters [ncells, 2]: distances between the
    centroids of the two end-vertex sets along the rest x and y axes."""
    (ax0, ax1), (tr0, tr1) = sets
    n = len(offsets) - 1
    idx = torch.as_tensor(np.asarray(offsets[:-1]), device=x.device)
    out = []
    for a, b_ in ((ax0, ax1), (tr0, tr1)):
        ia = idx[:, None] + torch.as_tensor(a, device=x.device)[None, :]
        ib = idx[:, None] + torch.as_tensor(b_, device=x.device)[None, :]
        ca = x[:, ia].mean(dim=2)     # [3, ncells]
        cb = x[:, ib].mean(dim=2)
        out.append(torch.sqrt(((cb - ca) ** 2).sum(dim=0)))
    return torch.stack(out, dim=1).reshape(n, 2)


class Calibration:
    """Membrane-parameter calibration against target diameters (the adjoint use case):
    loss = sum over cells of (D_ax - T_ax)^2 + (D_tr - T_tr)^2 after an nsteps rollout.
    Holds one homogeneous FP64 batch; `rebuild(weights)` refactors the type."""

    def __init__(self, mesh, material, dt: float, ncells: int):
        self.mesh, self.dt, self.ncells = mesh, dt, ncells
        self.sets = end_vertex_sets(mesh.verts)
        self.rebuild(np.asarray(material, dtype=np.float64))

    def rebuild(self, weights: np.ndarray):
        self.material = tuple(float(w) for w in weights[:4]) + (float(weights[4]) if len(weights) > 4 else 1.1,)
        self.types = [native.CellType(self.mesh.verts, self.mesh.tris, self.material, self.dt)]
        self.batch = native.Batch(self.types, np.zeros(self.ncells, np.int32), native.FP64)
        self.offsets = self.batch.offsets

    def loss(self, x0, v0, f, targets, iters, nsteps, ckpt_every):
        w = torch.tensor([self.material[:4]], dtype=torch.float64, device=x0.device, requires_grad=True)
        toc = torch.zeros(self.ncells, dtype=torch.int32, device=x0.device)
        xN, _ = rollout(self.batch, x0, v0, f, w, toc, iters, nsteps, ckpt_every)
        D = diameters(xN, self.offsets, self.sets)
        return ((D - targets) ** 2).sum(), w
