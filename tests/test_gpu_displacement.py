"""GPU parity of the displacement at the voxel corners (Eq. Fsplit), its transpose and the
gradient of a displacement-mismatch loss through the coupled adjoint, against the oracle.
Collected after the other GPU tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fg_oracle as O
from oracle import fg_oracle_adjoint as A
from paper_2411_16583_gb300 import binding as B, synth as S
from tests.helpers import oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available()
    return B.load_library()


@pytest.mark.parametrize("shape", [(8, 12, 16), (1, 64, 64), (24, 48, 80)])
def test_displacement_matches_oracle(lib, shape):
    """Corner displacement of a random F and Fbar, and the transpose of a random r, on the
    device against the oracle (FP64)."""
    rng = np.random.default_rng(5)
    ph = S.default_phases()
    pid = S.random_phase_map(shape, 1)
    h = (1.0e-7, 1.1e-7, 0.9e-7)
    sol = B.Solver(shape, h, ph, pid, np.zeros(shape), lib=lib)
    prm = oracle_params(ph, pid, h)
    F = np.eye(3).reshape(3, 3, 1, 1, 1) + 0.02 * rng.standard_normal((3, 3) + shape)
    Fbar = np.eye(3) + 0.01 * rng.standard_normal((3, 3))
    assert rel_err(sol.displacement(F, Fbar), A.corner_displacement(F, Fbar, prm)) < 1e-12
    r = rng.standard_normal((3,) + shape)
    assert rel_err(sol.displacement_adjoint(r), A.corner_displacement_adjoint(r, prm)) < 1e-12
    sol.close()


def test_displacement_mismatch_gradient_matches_oracle(lib):
    """d/dlog(E, D) of a displacement-mismatch loss after two damaging steps, through torch
    autograd on the device (CoupledSteps, then Displacement), against the oracle's adjoint;
    the toughness gradient vanishes on both sides (g_c cancels from the phase field)."""
    from paper_2411_16583_gb300.autograd import coupled_steps, displacement_mismatch
    from tests.test_oracle_adjoint import _strength_disc
    shape, logs, ls, src, prm, phases, pid = _strength_disc()
    tols = dict(tol_newton=1e-12, tol_cg=1e-13, tol_chem=1e-12, tol_chem_cg=1e-13,
                tol_pff_cg=1e-13, tol_stag=1e-10, max_stag=400)
    w = S.Workload(name="strength_disc12", shape=shape, h=(1e-7,) * 3, phases=phases,
                   phase_id=pid.astype(np.uint8), cdot_B=src, c_init=np.full(shape, 0.01),
                   gc=1.0, lc=2e-7, dt=1.0, nsteps=2, log_smax=ls)
    w.tol = tols
    rng = np.random.default_rng(8)
    u_obs = 1e-10 * rng.standard_normal((3,) + shape)
    wt = rng.uniform(0.0, 1.0, shape)
    geo = B.Solver(shape, w.h, phases, pid, np.zeros(shape), lib=lib)
    t = [torch.tensor(x, requires_grad=True) for x in logs]
    c, F, d = coupled_steps(*t, dict(w=w, nsteps=2, lib=lib, ckpt=1))
    L = displacement_mismatch(F, np.eye(3), torch.from_numpy(u_obs), torch.from_numpy(wt), geo)
    L.backward()
    tol = O.Tolerances(**tols)
    traj = A.forward(prm, np.full(shape, 0.01), src, [1.0, 1.0], [np.eye(3)] * 2, tol)
    Lr, seedF = A.displacement_mismatch(traj[-1].F, np.eye(3), u_obs, wt, prm)
    z = np.zeros(shape)
    g, _ = A.adjoint(prm, traj, [1.0, 1.0], dict(c=z, F=seedF, d=z, H=z), tol)
    assert traj[-1].d.max() > 0.5
    assert abs(L.item() - Lr) <= 1e-8 * Lr
    scale = max(np.abs(g[k]).max() for k in g)
    assert np.abs(t[1].grad.numpy()).max() < 1e-12 * scale
    for k, ti in (("E", t[0]), ("D", t[2])):
        assert np.abs(ti.grad.numpy() - g[k]).max() < 1e-8 * scale, k
    geo.close()
