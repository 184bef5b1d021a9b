"""torch.autograd.Functions over the C ABI with the hand-written adjoints as backward.

MechEquilibrium: F(log E) of the mechanical equilibrium (Alg. 1) at fixed (c, d);
  backward solves G K G lambda = G dL/dF (fg_adjoint_mech), dL/dlogE = -lambda : P.
CoupledSteps: the final state (c, F, d) after n staggered steps (Alg. 4) as a function of
  the per-voxel log E, log g_c, log D (a per-voxel strength of the workload is a fixed
  input); backward runs the recorded steps in reverse
  (fg_tape_begin / fg_adjoint with the seeds dL/d(c, F, d)).
Everything runs in the CUDA library; this module only moves arguments.
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


class CoupledSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, logE, loggc, logD, spec):
        """spec: dict with a ``synth.Workload`` ``w``, ``nsteps`` and optional ``ckpt``
        (steps per checkpoint), ``lib``, ``precision``, ``opts``.  Returns (c, F, d)."""
        w = spec["w"]
        np_ = lambda t: t.detach().double().cpu().numpy()
        sol = B.Solver(w.shape, w.h, w.phases, w.phase_id, w.cdot_B, c_init=w.c_init,
                       log_E=np_(logE), log_gc=np_(loggc), log_D=np_(logD),
                       log_smax=w.log_smax, lib=spec.get("lib"),
                       precision=spec.get("precision", B.FG_FP64), gc=w.gc, lc=w.lc, RT=w.RT,
                       cmax=w.cmax, **{**w.tol, **spec.get("opts", {})})
        sol.tape(spec.get("ckpt", 1))
        for _ in range(spec["nsteps"]):
            sol.step(w.dt)
        ctx.sol = sol
        dev = logE.device
        return (torch.from_numpy(sol.get(B.FIELD_C)).to(dev),
                torch.from_numpy(sol.get(B.FIELD_F)).to(dev),
                torch.from_numpy(sol.get(B.FIELD_D)).to(dev))

    @staticmethod
    def backward(ctx, gc, gF, gd):
        np_ = lambda t: None if t is None else t.detach().double().contiguous().cpu().numpy()
        _, g, _ = ctx.sol.adjoint(B.FG_LOSS_SEEDS, seed_c=np_(gc), seed_F=np_(gF), seed_d=np_(gd))
        ctx.sol.close()
        dev = (gc if gc is not None else gF if gF is not None else gd).device
        return (torch.from_numpy(g["E"]).to(dev), torch.from_numpy(g["gc"]).to(dev),
                torch.from_numpy(g["D"]).to(dev), None)


def coupled_steps(logE, loggc, logD, spec):
    return CoupledSteps.apply(logE, loggc, logD, spec)
