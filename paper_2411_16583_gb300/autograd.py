"""torch.autograd.Function over the C ABI: mechanical equilibrium F(log E) with the
hand-written adjoint as its backward.

forward:  builds a context with the per-voxel log stiffness, sets (c, d) and solves
          Alg. 1 (fg_solve_mech); returns the converged deformation gradient F.
backward: for dL/dF from autograd, fg_adjoint_mech solves G K G lambda = G dL/dF with the
          fused mechanical CG and returns dL/dlogE = -lambda : P.
Both run entirely in the CUDA library; this module only moves arguments.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class MechEquilibrium(torch.autograd.Function):
    @staticmethod
    def forward(ctx, logE, spec):
        """spec: dict with shape, h, phases, phase_id, c, d and optional Fbar, lib, opts."""
        sol = B.Solver(spec["shape"], spec["h"], spec["phases"], spec["phase_id"],
                       np.zeros(spec["shape"]), log_E=logE.detach().double().cpu().numpy(),
                       lib=spec.get("lib"), **spec.get("opts", {}))
        sol.set(B.FIELD_C, spec["c"])
        sol.set(B.FIELD_D, spec["d"])
        sol.solve_mech(spec.get("Fbar"))
        F = torch.from_numpy(sol.get(B.FIELD_F)).to(logE.device)
        ctx.sol = sol
        return F

    @staticmethod
    def backward(ctx, gF):
        g, _ = ctx.sol.adjoint_mech(gF.detach().double().contiguous().cpu().numpy())
        ctx.sol.close()
        return torch.from_numpy(g).to(gF.device), None


def mech_equilibrium(logE, spec):
    return MechEquilibrium.apply(logE, spec)
