"""torch.autograd.Functions over the C ABI with the hand-written adjoints as backward.

MechEquilibrium: F(log E) of the mechanical equilibrium (Alg. 1) at fixed (c, d);
  backward solves G K G lambda = G dL/dF (fg_adjoint_mech), dL/dlogE = -lambda : P.
Displacement: the displacement at the voxel corners as a function of F (Eq. Fsplit;
  fg_displacement), backward by the transpose (fg_displacement_adjoint); with
  CoupledSteps it gives the gradient of a displacement-mismatch loss.
CoupledSteps: the final state (c, F, d) after n staggered steps (Alg. 4) as a function of
  the per-voxel log E, log g_c, log D (a per-voxel strength of the workload is a fixed
  input); backward runs the recorded steps in reverse
  (fg_tape_begin / fg_adjoint with the seeds dL/d(c, F, d)).
Everything runs in the CUDA library; this module only moves arguments.  Outputs, seeds
and gradients of tensors on a CUDA device stay on the device (the library reads and writes
device pointers); only the set-up inputs of a context (the per-voxel log fields) are read
from host memory, as fg_setup takes them.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def _field(sol, field, device):
    """A stored field as a tensor on `device` (copied device to device on a GPU)."""
    if device.type == "cuda":
        return sol.get(field, device=device)
    return torch.from_numpy(sol.get(field))


def _pass(t):
    """A tensor argument for the library: the CUDA tensor itself, else a host array."""
    if t is None:
        return None
    t = t.detach()
    return t.double().contiguous() if t.is_cuda else t.double().contiguous().numpy()


def _back(g, device):
    return g if torch.is_tensor(g) else torch.from_numpy(g).to(device)


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
        F = _field(sol, B.FIELD_F, logE.device)
        ctx.sol = sol
        return F

    @staticmethod
    def backward(ctx, gF):
        g, _ = ctx.sol.adjoint_mech(_pass(gF))
        ctx.sol.close()
        return _back(g, gF.device), None


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
        return (_field(sol, B.FIELD_C, dev), _field(sol, B.FIELD_F, dev),
                _field(sol, B.FIELD_D, dev))

    @staticmethod
    def backward(ctx, gc, gF, gd):
        _, g, _ = ctx.sol.adjoint(B.FG_LOSS_SEEDS, seed_c=_pass(gc), seed_F=_pass(gF),
                                  seed_d=_pass(gd))
        ctx.sol.close()
        dev = (gc if gc is not None else gF if gF is not None else gd).device
        return _back(g["E"], dev), _back(g["gc"], dev), _back(g["D"], dev), None


def coupled_steps(logE, loggc, logD, spec):
    return CoupledSteps.apply(logE, loggc, logD, spec)


class Displacement(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, Fbar, sol):
        """F (3, 3, nz, ny, nx) -> u (3, nz, ny, nx) at the voxel corners, u = (Fbar - I) x
        + u~ with grad u~ = F - Fbar; Fbar (3, 3) is a fixed input.  sol is any
        ``binding.Solver`` on the same grid (only its transforms are used)."""
        u = sol.displacement(_pass(F), np.asarray(Fbar, dtype=float))
        ctx.sol = sol
        return _back(u, F.device)

    @staticmethod
    def backward(ctx, gu):
        g = ctx.sol.displacement_adjoint(_pass(gu))
        return _back(g, gu.device), None, None


def displacement(F, Fbar, sol):
    return Displacement.apply(F, Fbar, sol)


def displacement_mismatch(F, Fbar, u_obs, w, sol):
    """L = 1/2 sum over the corners of w |u - u_obs|^2 h^3, u = displacement(F, Fbar, sol);
    u_obs (3, nz, ny, nx) and w (nz, ny, nx) are tensors."""
    u = displacement(F, Fbar, sol)
    h3 = sol.h[0] * sol.h[1] * sol.h[2]
    diff = u - u_obs
    return 0.5 * h3 * (w * diff * diff).sum()

