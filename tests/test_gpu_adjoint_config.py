"""The coupled adjoint on the particle workload with per-voxel log fields: at the full 128^3
size against central differences of the GPU forward, and on a reduced 3D grid against the
oracle's adjoint.  The loss is a seeded random linear functional of the final (c, F, d)
(FG_LOSS_SEEDS): the rough-ellipsoid particle does not crack in its first steps, so its
fracture energy and the toughness gradient are zero there (the fracture-energy loss is
checked on the damaging disc in test_gpu_parity.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fg_oracle as O
from oracle import fg_oracle_adjoint as A
from paper_2411_16583_gb300 import binding as B, synth as S
from tests.helpers import oracle_params, rel_err

pytestmark = pytest.mark.gpu

# the forward's tolerances for differencing: Newton 1e-12 and Krylov 1e-13 (at Newton 1e-13
# the FP64 oracle's mechanical Newton stalls on the rough particle in its round-off floor)
TIGHT = dict(tol_newton=1e-12, tol_cg=1e-13, tol_chem=1e-12, tol_chem_cg=1e-13,
             tol_pff_cg=1e-13, tol_stag=1e-12, max_stag=400)


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available()
    return B.load_library()


def _particle(n):
    """The 128^3 rough-ellipsoid recipe scaled to n^3 with per-voxel log E, log g_c, log D
    ~ N(0, 0.1^2)."""
    f = n / 128
    w = S.ellipsoid(n=n, axes=(50 * f, 40 * f, 35 * f), rough_std=1.5 * f, rough_corr=4 * f,
                    band=max(1, round(8 * f)), nsteps=50)
    return S.with_log_fields(w, std=0.1)


def _seeds(shape, seed=3):
    rng = np.random.default_rng(seed)
    return dict(c=rng.standard_normal(shape), F=rng.standard_normal((3, 3) + shape),
                d=rng.standard_normal(shape))


def _loss(sol, s):
    return float(np.sum(s["c"] * sol.get(B.FIELD_C)) + np.sum(s["F"] * sol.get(B.FIELD_F))
                 + np.sum(s["d"] * sol.get(B.FIELD_D)))


def test_adjoint_128_matches_central_differences(lib):
    """128^3, one step, the hand-written FP64 reverse pass: the gradient with respect to log E
    and log D at 32 seeded particle voxels (16 each) against central differences of the
    forward at h = 1e-6, and at 8 of them also at h = 1e-4.  The differenced forwards run in
    the mixed form at Newton 1e-12 / Krylov 1e-13 (the same converged solution map as the
    FP64 form; a forward takes about a second instead of ten).  At h = 1e-6 the difference
    quotient of a loss summed over 2 M voxels carries solver noise of order 1e-4 of the
    largest gradient entry (measured: up to 5e-4 at single voxels, FP64 or mixed forwards);
    at h = 1e-4 that noise is 100 times smaller while the truncation error (h^2) stays far
    below it, so there the bar is tight.  The toughness
    gradient is 0 (no damage; g_c(x) cancels from the phase field as the history carries
    it).  The chaining of steps through checkpoints is checked on the 32^3 sphere of
    test_gpu_parity.py."""
    w = _particle(128)
    nsteps = 1
    s = _seeds(w.shape)
    sol = B.from_workload(w, lib=lib, **TIGHT)
    sol.tape(1)
    for _ in range(nsteps):
        sol.step(w.dt)
    _, g, st = sol.adjoint(B.FG_LOSS_SEEDS, seed_c=s["c"], seed_F=s["F"], seed_d=s["d"])
    sol.close()
    assert st["steps"] == nsteps
    assert np.abs(g["gc"]).max() <= 1e-12 * np.abs(g["E"]).max()
    rng = np.random.default_rng(7)
    inside = np.flatnonzero(w.phase_id.ravel() == 0)
    picks = {"E": rng.choice(inside, 16, replace=False), "D": rng.choice(inside, 16, replace=False)}

    def loss_with(field, v, dx):
        logs = {"E": w.log_E.copy(), "D": w.log_D.copy()}
        logs[field].flat[v] += dx
        x = B.Solver(w.shape, w.h, w.phases, w.phase_id, w.cdot_B, c_init=w.c_init,
                     log_E=logs["E"], log_D=logs["D"], log_gc=w.log_gc, lib=lib, gc=w.gc,
                     lc=w.lc, precision=B.FG_MIXED, **{**w.tol, **TIGHT})
        for _ in range(nsteps):
            x.step(w.dt)
        val = _loss(x, s)
        x.close()
        return val

    scale = {k: np.abs(g[k]).max() for k in ("E", "D")}
    errs, errs_wide = [], []
    for field, vox in picks.items():
        for j, v in enumerate(vox):
            fd = (loss_with(field, v, 1e-6) - loss_with(field, v, -1e-6)) / 2e-6
            errs.append((field, int(v), abs(fd - g[field].flat[v]) / scale[field]))
            if j < 4:
                fd = (loss_with(field, v, 1e-4) - loss_with(field, v, -1e-4)) / 2e-4
                errs_wide.append((field, int(v), abs(fd - g[field].flat[v]) / scale[field]))
    assert max(e for _, _, e in errs_wide) <= 2e-5, (errs_wide, errs)
    assert max(e for _, _, e in errs) <= 1e-3, errs
    assert np.median([e for _, _, e in errs]) <= 3e-4, errs


def test_adjoint_reduced_3d_matches_oracle(lib):
    """The same recipe at 16^3: two FP64 steps and the reverse pass against the oracle's
    adjoint (all three gradients, to 1e-6 of their largest entry)."""
    w = _particle(16)
    nsteps = 2
    s = _seeds(w.shape)
    prm = oracle_params(w)
    tol = O.Tolerances(**{**{k: v for k, v in w.tol.items() if hasattr(O.Tolerances, k)}, **TIGHT})
    traj = A.forward(prm, w.c_init, w.cdot_B, [w.dt] * nsteps, [np.eye(3)] * nsteps, tol)
    z = np.zeros(w.shape)
    g_ref, _ = A.adjoint(prm, traj, [w.dt] * nsteps, dict(c=s["c"], F=s["F"], d=s["d"], H=z), tol)
    sol = B.from_workload(w, lib=lib, **TIGHT)
    sol.tape(1)
    for _ in range(nsteps):
        sol.step(w.dt)
    assert rel_err(sol.get(B.FIELD_F), traj[-1].F) < 1e-10
    _, g, _ = sol.adjoint(B.FG_LOSS_SEEDS, seed_c=s["c"], seed_F=s["F"], seed_d=s["d"])
    sol.close()
    for k in ("E", "D"):
        assert rel_err(g[k], g_ref[k]) < 1e-6, k
    scale = max(np.abs(g_ref[k]).max() for k in ("E", "D"))
    assert np.abs(g["gc"]).max() <= 1e-12 * scale and np.abs(g_ref["gc"]).max() <= 1e-12 * scale
