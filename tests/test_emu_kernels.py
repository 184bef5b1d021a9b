"""CPU checks of the CUDA kernel source through its host-emulation build.

``libfg_emu.so`` compiles the same kernel and runtime sources with FG_EMU: every block of
every kernel runs on the host, thread by thread between barriers.  These tests catch
indexing, tiling and FFT-plan mistakes without a GPU; the product path never loads this
library, and the parity that counts is the one of ``test_gpu_parity.py``.
"""
import numpy as np
import pytest

from oracle import fg_oracle as O
from paper_2411_16583_gb300 import binding as B, build, synth as S
from tests.helpers import (TOL_APPLY_FP32, TOL_APPLY_FP64, homogeneous_stretch_damage,
                           oracle_params, rel_err)

H3 = (1.0e-7, 1.1e-7, 0.9e-7)


@pytest.fixture(scope="module")
def emu():
    return B.load_library(build.build_emu())


# (64, 16, 16), (256, 8, 8), (8, 256, 8): the register-direct Y and Z passes (64 = 8 x 8,
# 256 = 16 x 16), including ragged row tiles; (8, 12, 16), (12, 8, 8), (48, 24, 8),
# (32, 48, 8): the same passes for two-stage plans of unequal radices (12 = 4 x 3,
# 24 = 8 x 3, 32 = 8 x 4, 48 = 16 x 3); (1, 8, 256): the X passes at the benchmark's row
# length
@pytest.mark.parametrize("shape", [(8, 12, 16), (1, 16, 24), (12, 8, 8), (64, 16, 16),
                                   (256, 8, 8), (8, 256, 8), (1, 64, 16), (1, 100, 100),
                                   (1, 8, 256), (48, 24, 8), (32, 48, 8)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("law", [S.LAW_NEOHOOKE, S.LAW_SVK])
def test_emulated_operators_match_oracle(emu, shape, prec, law):
    pid = S.random_phase_map(shape, 1)
    phases = S.default_phases(law=law)
    phases[1].E = 2e9
    sol = B.Solver(shape, H3, phases, pid, np.zeros(shape), lib=emu,
                   precision=B.FG_MIXED if prec else B.FG_FP64)
    F, c, d = S.random_state(shape, seed=2)
    Hh = np.random.default_rng(5).uniform(0, 1e6, shape)
    for f, v in ((B.FIELD_F, F), (B.FIELD_C, c), (B.FIELD_D, d), (B.FIELD_H, Hh)):
        sol.set(f, v)
    prm = oracle_params(phases, pid, H3)
    F = F.reshape((3, 3) + shape)
    dt_ = np.float32 if prec else np.float64
    tol = TOL_APPLY_FP32 if prec else TOL_APPLY_FP64
    x9 = S.random_tensor_field(shape, 3).astype(dt_)
    x1 = S.random_tensor_field(shape, 4, ncomp=1)[0].astype(dt_)
    y9, y1 = np.zeros_like(x9), np.zeros_like(x1)
    sol.apply(B.OP_MECH, x9, y9, prec)
    assert rel_err(y9.reshape(F.shape), O.mech_apply(F, c, d, prm, x9.astype(float).reshape(F.shape))) < tol
    sol.apply(B.OP_PFF, x1, y1, prec)
    assert rel_err(y1, O.pff_apply(x1.astype(float), Hh, prm)) < tol
    sol.apply(B.OP_PFF_PREC, x1, y1, prec)
    assert rel_err(y1, O.pff_precond(x1.astype(float), Hh.mean(), prm)) < tol
    sol.apply(B.OP_CHEM, x1, y1, prec, dt=0.7)
    ref = O.chem_apply(x1.astype(float), 1 / (c * (1 - c)), O.chem_conductivity(F, c, d, prm), 0.7, prm)
    assert rel_err(y1, ref) < tol
    assert rel_err(sol.get(B.FIELD_P), O.stress(F, c, d, prm)) < 1e-13
    sol.close()


@pytest.mark.parametrize("law", [S.LAW_NEOHOOKE, S.LAW_SVK])
def test_emulated_step_law(emu, law):
    """One coupled step of a small disc with each law against the oracle."""
    w = S.disc2d(n=16, radius=6.0, band=3, nsteps=10)
    w.phases = S.default_phases(law=law)
    prm = oracle_params(w)
    ref = O.CoupledState(prm, w.c_init, w.cdot_B)
    ref.step(w.dt, np.eye(3))
    sol = B.from_workload(w, lib=emu)
    sol.step(w.dt)
    assert rel_err(sol.get(B.FIELD_F), ref.F) < 1e-10
    assert rel_err(sol.get(B.FIELD_C), ref.c) < 1e-10
    sol.close()


def test_emulated_coupled_step_matches_oracle(emu):
    w = S.disc2d(n=16, radius=6.0, band=3, nsteps=10)
    prm = oracle_params(w)
    ref = O.CoupledState(prm, w.c_init, w.cdot_B)
    sol = B.from_workload(w, lib=emu)
    for _ in range(2):
        ref.step(w.dt, np.eye(3))
        st = sol.step(w.dt)
        assert abs(st["mass_err"]) < 1e-13
    assert rel_err(sol.get(B.FIELD_F), ref.F) < 1e-10
    assert rel_err(sol.get(B.FIELD_C), ref.c) < 1e-10
    em, ec, mass = sol.residual()
    assert em <= 1e-9 and ec < 1e-9
    assert abs(mass - ref.c.sum()) < 1e-10 * mass
    sol.close()


def test_emulated_mixed_step_close_to_fp64(emu):
    w = S.disc2d(n=16, radius=6.0, band=3, nsteps=10)
    a = B.from_workload(w, lib=emu)
    b = B.from_workload(w, lib=emu, precision=B.FG_MIXED)
    for _ in range(2):
        a.step(w.dt)
        b.step(w.dt)
    assert rel_err(b.get(B.FIELD_F), a.get(B.FIELD_F)) < 1e-7
    assert rel_err(b.get(B.FIELD_C), a.get(B.FIELD_C)) < 1e-7
    a.close()
    b.close()


def test_emulated_batch_equals_solo_runs(emu):
    """A batch of RVEs of uneven sizes stepped together gives each member's solo result."""
    ws = [S.sphere(n, r, band=2, nsteps=10, seed=i) for i, (n, r) in enumerate([(8, 0.3), (12, 0.4), (16, 0.35)])]
    solo = [B.from_workload(w, lib=emu) for w in ws]
    for s, w in zip(solo, ws):
        s.step(w.dt)
    members = [B.from_workload(w, lib=emu) for w in ws]
    batch = B.Batch(members)
    stats = batch.step(1.0)
    assert all(st["status"] == 0 for st in stats)
    for a, b in zip(members, solo):
        np.testing.assert_array_equal(a.get(B.FIELD_F), b.get(B.FIELD_F))
        np.testing.assert_array_equal(a.get(B.FIELD_C), b.get(B.FIELD_C))
    batch.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_emulated_grouped_batch_apply_equals_member_applies(emu, prec):
    """fg_batch_apply runs each pass once over every member of equal grid (block m P + b of
    a grouped launch is block b of member m, arguments from a device table): each member's
    result is bit for bit its own fg_apply, in fewer launches; members of three grids form
    three groups (two equal-grid members share one)."""
    ws = [S.sphere(n, r, band=2, nsteps=10, seed=i)
          for i, (n, r) in enumerate([(8, 0.3), (12, 0.4), (8, 0.35), (16, 0.3)])]
    members = [B.from_workload(w, lib=emu, precision=B.FG_MIXED) for w in ws]
    rng = np.random.default_rng(3)
    dt = np.float32 if prec == 1 else np.float64
    for m, w in zip(members, ws):  # a state away from the identity
        F = m.get(B.FIELD_F)
        m.set(B.FIELD_F, F + 0.01 * rng.standard_normal(F.shape))
    xs = [rng.standard_normal((9,) + w.shape).astype(dt) for w in ws]
    solo = []
    l0 = B.kernel_launches(emu)
    for m, x in zip(members, xs):
        y = np.zeros_like(x)
        m.apply(B.OP_MECH, x, y, prec)
        solo.append(y)
    l_solo = B.kernel_launches(emu) - l0
    batch = B.Batch(members)
    ys = [np.zeros_like(x) for x in xs]
    l0 = B.kernel_launches(emu)
    batch.apply(xs, ys, prec)
    l_batch = B.kernel_launches(emu) - l0
    for y, ref in zip(ys, solo):
        np.testing.assert_array_equal(y, ref)
        assert np.abs(ref).max() > 0
    # per member: its state build and its passes; grouped: the state builds, then one
    # launch per pass and group
    passes = (l_solo - l_batch) // (len(ws) - 3)
    assert l_batch < l_solo and passes >= 5
    with pytest.raises(B.FgError):
        batch.apply(xs, ys, prec, op=B.OP_PFF)
    batch.close()


def test_emulated_grouped_batch_apply_keeps_member_settings(emu):
    """Members of one grid that differ in law (Saint-Venant-Kirchhoff against Neo-Hookean)
    run in separate groups, and a member under mixed stress control keeps its projection
    (the kept zero modes): every result is still bit for bit the member's own fg_apply."""
    ws = [S.sphere(8, 0.3, band=2, nsteps=10, seed=0),
          S.sphere(8, 0.35, band=2, nsteps=10, seed=1, phases=S.default_phases(law=S.LAW_SVK)),
          S.sphere(8, 0.4, band=2, nsteps=10, seed=2)]
    members = [B.from_workload(w, lib=emu, precision=B.FG_MIXED) for w in ws]
    mask = np.zeros((3, 3), dtype=bool)
    mask[1, 1] = mask[0, 2] = True
    members[2].stress_control(mask, np.zeros((3, 3)))
    rng = np.random.default_rng(4)
    xs = [rng.standard_normal((9,) + w.shape).astype(np.float32) for w in ws]
    solo = []
    for m, x in zip(members, xs):
        y = np.zeros_like(x)
        m.apply(B.OP_MECH, x, y, 1)
        solo.append(y)
    batch = B.Batch(members)
    ys = [np.zeros_like(x) for x in xs]
    l0 = B.kernel_launches(emu)
    batch.apply(xs, ys, 1)
    l_batch = B.kernel_launches(emu) - l0
    for y, ref in zip(ys, solo):
        np.testing.assert_array_equal(y, ref)
    members[2].stress_control(None)
    y_free = np.zeros_like(xs[2])
    members[2].apply(B.OP_MECH, xs[2], y_free, 1)
    assert np.abs(y_free - ys[2]).max() > 0  # the mask changed that member's result
    batch.close()
    assert l_batch > 0


@pytest.mark.parametrize("law", [S.LAW_NEOHOOKE, S.LAW_SVK])
def test_emulated_mech_adjoint_matches_oracle(emu, law):
    shape = (8, 8, 16)
    rng = np.random.default_rng(9)
    pid = S.random_phase_map(shape, 2)
    phases = S.default_phases(law=law)
    phases[1].E = 2e9
    logE = rng.normal(0, 0.1, shape)
    c = rng.uniform(0.05, 0.4, shape)
    d = rng.uniform(0.0, 0.3, shape)
    sol = B.Solver(shape, H3, phases, pid, np.zeros(shape), log_E=logE, lib=emu,
                   tol_newton=1e-13, tol_cg=1e-14)
    sol.set(B.FIELD_C, c)
    sol.set(B.FIELD_D, d)
    sol.solve_mech()
    F = sol.get(B.FIELD_F)
    prm = O.make_params([O.Phase(**vars(p)) for p in phases], pid, H3, gc=1.0, lc=2e-7, log_E=logE)
    _, err = O.mech_residual(F, c, d, prm, np.eye(3))
    assert err < 1e-12
    W = rng.standard_normal((3, 3) + shape)
    g, it = sol.adjoint_mech(W)
    ref = O.mech_adjoint(F, c, d, prm, W, 1e-14, 2000)
    assert it > 0 and rel_err(g, ref) < 1e-9
    sol.close()


def test_emulated_damage_with_log_fields_matches_oracle(emu):
    """Two steps of a 12 x 12 disc whose second step damages, with per-voxel log E, log D
    and log g_c: the history H = max(H_t, g_c(x)/(2 l_c) D_f) and the phase field solved
    with H g_c/g_c(x) against the oracle."""
    from tests.test_oracle_adjoint import _disc
    shape, logs, src, _, prm_of, phases, pid = _disc(n=12, smax=21e6)
    prm = prm_of(*logs)
    tols = dict(tol_newton=1e-12, tol_stag=1e-10, max_stag=400)
    ref = O.CoupledState(prm, np.full(shape, 0.01), src, O.Tolerances(**tols))
    sol = B.Solver(shape, (1e-7,) * 3, phases, pid, src, c_init=np.full(shape, 0.01),
                   log_E=logs[0], log_gc=logs[1], log_D=logs[2], lib=emu, gc=1.0, lc=2e-7,
                   **tols)
    for _ in range(2):
        ref.step(1.0, np.eye(3))
        sol.step(1.0)
    assert ref.d.max() > 0.01
    assert rel_err(sol.get(B.FIELD_F), ref.F) < 1e-8
    assert rel_err(sol.get(B.FIELD_C), ref.c) < 1e-8
    assert rel_err(sol.get(B.FIELD_H), ref.H) < 1e-8
    assert np.abs(sol.get(B.FIELD_D) - ref.d).max() < 1e-8
    sol.close()


def test_emulated_per_voxel_strength_matches_oracle(emu):
    """Two steps of the disc with per-voxel log E, log D, log g_c and a Gumbel-distributed
    strength sigma_max(x) (Sec. 5.1): damage starts at the weak voxels in the first step;
    F, c, H and d against the oracle."""
    from tests.test_oracle_adjoint import _strength_disc
    shape, logs, ls, src, prm, phases, pid = _strength_disc()
    tols = dict(tol_newton=1e-12, tol_stag=1e-10, max_stag=400)
    ref = O.CoupledState(prm, np.full(shape, 0.01), src, O.Tolerances(**tols))
    sol = B.Solver(shape, (1e-7,) * 3, phases, pid, src, c_init=np.full(shape, 0.01),
                   log_E=logs[0], log_gc=logs[1], log_D=logs[2], log_smax=ls, lib=emu, gc=1.0,
                   lc=2e-7, **tols)
    ref.step(1.0, np.eye(3))
    sol.step(1.0)
    assert ref.d.max() > 0.01  # damaging already
    ref.step(1.0, np.eye(3))
    sol.step(1.0)
    assert rel_err(sol.get(B.FIELD_F), ref.F) < 1e-8
    assert rel_err(sol.get(B.FIELD_C), ref.c) < 1e-8
    assert rel_err(sol.get(B.FIELD_H), ref.H) < 1e-8
    assert np.abs(sol.get(B.FIELD_D) - ref.d).max() < 1e-8
    sol.close()


def test_emulated_adjoint_with_per_voxel_strength_matches_oracle(emu):
    """dGamma_E/dlog(E, g_c, D) of the CUDA reverse pass with a per-voxel strength (a fixed
    input) against the oracle's adjoint, two damaging steps."""
    from oracle import fg_oracle_adjoint as A
    from tests.test_oracle_adjoint import _strength_disc
    shape, logs, ls, src, prm, phases, pid = _strength_disc()
    tols = dict(tol_newton=1e-12, tol_cg=1e-13, tol_chem=1e-12, tol_chem_cg=1e-13,
                tol_pff_cg=1e-13, tol_stag=1e-10, max_stag=400)
    val, g = A.crack_energy_gradient(prm, np.full(shape, 0.01), src, [1.0, 1.0],
                                     [np.eye(3)] * 2, O.Tolerances(**tols))
    sol = B.Solver(shape, (1e-7,) * 3, phases, pid, src, c_init=np.full(shape, 0.01),
                   log_E=logs[0], log_gc=logs[1], log_D=logs[2], log_smax=ls, lib=emu, gc=1.0,
                   lc=2e-7, **tols)
    sol.tape(1)
    for _ in range(2):
        sol.step(1.0)
    v2, g2, _ = sol.adjoint()
    assert abs(v2 - val) < 1e-8 * val
    assert np.abs(g["gc"]).max() > 0.0
    for k in ("E", "gc", "D"):
        assert rel_err(g2[k], g[k]) < 1e-9, k
    sol.close()


@pytest.mark.parametrize("ckpt", [1, 2])
def test_emulated_coupled_adjoint_matches_oracle(emu, ckpt):
    """dGamma_E/dlog(E, g_c, D) of the CUDA reverse pass (tape, recompute from
    checkpoints, transposed block sweeps with GMRES, chemistry transpose) against the
    oracle's adjoint, on two steps of a 12 x 12 disc whose second step damages."""
    from oracle import fg_oracle_adjoint as A
    from tests.test_oracle_adjoint import _disc
    shape, logs, src, _, prm_of, phases, pid = _disc(n=12, smax=21e6)
    prm = prm_of(*logs)
    tols = dict(tol_newton=1e-12, tol_cg=1e-13, tol_chem=1e-12, tol_chem_cg=1e-13,
                tol_pff_cg=1e-13, tol_stag=1e-10, max_stag=400)
    val, g = A.crack_energy_gradient(prm, np.full(shape, 0.01), src, [1.0, 1.0],
                                     [np.eye(3)] * 2, O.Tolerances(**tols))
    sol = B.Solver(shape, (1e-7,) * 3, phases, pid, src, c_init=np.full(shape, 0.01),
                   log_E=logs[0], log_gc=logs[1], log_D=logs[2], lib=emu, gc=1.0, lc=2e-7,
                   **tols)
    sol.tape(ckpt)
    for _ in range(2):
        sol.step(1.0)
    d_before = sol.get(B.FIELD_D)
    v2, g2, st = sol.adjoint()
    assert st["steps"] == 2 and st["gmres"] >= 1
    assert st["recomputed"] == 2
    assert abs(v2 - val) < 1e-8 * val
    for k in ("E", "gc", "D"):
        assert rel_err(g2[k], g[k]) < 1e-9, k
    np.testing.assert_array_equal(sol.get(B.FIELD_D), d_before)  # state restored
    sol.close()


def test_emulated_coupled_steps_autograd(emu):
    """torch autograd through CoupledSteps: the gradient of a loss on the final (c, F, d)
    equals the one fg_adjoint returns for the same seeds, and a directional derivative
    of the loss agrees with central differences of the forward."""
    import torch
    from paper_2411_16583_gb300.autograd import coupled_steps
    from tests.test_oracle_adjoint import _disc
    shape, logs, src, _, prm_of, phases, pid = _disc(n=12, smax=21e6)
    w = S.Workload(name="disc12", shape=shape, h=(1e-7,) * 3, phases=phases,
                   phase_id=pid.astype(np.uint8), cdot_B=src, c_init=np.full(shape, 0.01),
                   gc=1.0, lc=2e-7, dt=1.0, nsteps=2)
    w.tol = dict(tol_newton=1e-12, tol_cg=1e-13, tol_chem=1e-12, tol_chem_cg=1e-13,
                 tol_pff_cg=1e-13, tol_stag=1e-10, max_stag=400)
    spec = dict(w=w, nsteps=2, lib=emu, ckpt=2)
    rng = np.random.default_rng(1)
    wc, wd = rng.standard_normal(shape), rng.standard_normal(shape)
    wF = rng.standard_normal((3, 3) + shape)

    def loss_of(lE, lG, lD):
        c, F, d = coupled_steps(lE, lG, lD, spec)
        return ((c * torch.from_numpy(wc)).sum() + (F * torch.from_numpy(wF)).sum()
                + (d * torch.from_numpy(wd)).sum())
    t = [torch.tensor(x, requires_grad=True) for x in logs]
    L = loss_of(*t)
    L.backward()
    h = 1e-4
    dirs = [0.3 * rng.standard_normal(shape) for _ in range(3)]
    with torch.no_grad():
        lp = loss_of(*[torch.tensor(x + h * dx) for x, dx in zip(logs, dirs)]).item()
        lm = loss_of(*[torch.tensor(x - h * dx) for x, dx in zip(logs, dirs)]).item()
    fd = (lp - lm) / (2 * h)
    adj = sum(float((ti.grad.numpy() * dx).sum()) for ti, dx in zip(t, dirs))
    assert abs(adj - fd) <= 1e-5 * abs(fd), (adj, fd)


def test_emulated_bimaterial_diffusion_100(emu):
    """A 100 x 100 bimaterial (transform length 100 = 4 x 5 x 5; diffusivities 100 times
    apart, no swelling) with an initial concentration step, two coupled steps against the
    oracle: the diffusion set-up of the paper's bimaterial validation on a
    non-power-of-two grid."""
    shape = (1, 100, 100)
    pid = np.zeros(shape, dtype=np.uint8)
    pid[..., 50:] = 1
    phases = [S.PhaseSpec(law=S.LAW_NEOHOOKE, E=10e9, nu=0.3, Omega=0.0, c0=0.01, D=1e-14,
                          sigma_max=100e6),
              S.PhaseSpec(law=S.LAW_NEOHOOKE, E=5e9, nu=0.3, Omega=0.0, c0=0.01, D=1e-16,
                          sigma_max=100e6)]
    c_init = np.full(shape, 0.05)
    c_init[:, 40:60, :] = 0.4
    h = (0.1e-6,) * 3
    w = S.Workload(name="bimaterial100", shape=shape, h=h, phases=phases, phase_id=pid,
                   cdot_B=np.zeros(shape), c_init=c_init, gc=1.0, lc=2e-7, dt=5.0, nsteps=2)
    prm = oracle_params(w)
    ref = O.CoupledState(prm, c_init, np.zeros(shape))
    sol = B.from_workload(w, lib=emu)
    for _ in range(2):
        ref.step(w.dt, np.eye(3))
        st = sol.step(w.dt)
        assert abs(st["mass_err"]) < 1e-13
    assert rel_err(sol.get(B.FIELD_C), ref.c) < 1e-10
    c = sol.get(B.FIELD_C)
    # the step runs along y; the slow phase (x >= 50) keeps more of its spread
    assert c[0, :, 80].std() > c[0, :, 10].std()
    sol.close()


def test_emulated_mixed_control_step_matches_oracle(emu):
    """One coupled step of a swelling particle in a buffer under mixed macroscopic control
    (F11 prescribed at 1.01, every other mean stress zero) against the oracle: fields and the
    solved mean deformation gradient."""
    w = S.disc2d(n=16, radius=6.0, band=3, nsteps=10)
    prm = oracle_params(w)
    mask = np.ones((3, 3), dtype=bool)
    mask[0, 0] = False
    prm.stress_mask, prm.Pbar = mask, np.zeros((3, 3))
    tols = dict(tol_newton=1e-12, tol_cg=1e-13, tol_stag=1e-11)  # compare beyond the stop
    ref = O.CoupledState(prm, w.c_init, w.cdot_B, O.Tolerances(**tols))
    Fbar = np.diag([1.01, 1.0, 1.0])
    ref.step(w.dt, Fbar)
    sol = B.from_workload(w, lib=emu, **tols)
    sol.stress_control(mask, np.zeros((3, 3)))
    sol.step(w.dt, Fbar)
    F = sol.get(B.FIELD_F)
    assert rel_err(F, ref.F) < 1e-9
    assert rel_err(sol.get(B.FIELD_C), ref.c) < 1e-10
    np.testing.assert_allclose(F.mean(axis=(2, 3, 4)), ref.Fbar, atol=1e-12)
    assert abs(ref.Fbar[1, 1] - 1.0) > 1e-4  # the lateral mean strain was solved for
    sol.close()


def test_emulated_full_chemistry_jacobian_matches_oracle(emu):
    """The chemistry Newton with the full Jacobian (chem_full_jacobian) on a 32 x 32 version
    of the Omega = 1.3 Saint-Venant-Kirchhoff Gumbel disc: one coupled step against the
    oracle's."""
    w = S.gumbel_disc(n=32, band=2, nsteps=20)
    prm = oracle_params(w)
    ref = O.CoupledState(prm, w.c_init, w.cdot_B, O.Tolerances(**w.tol))
    st_ref = ref.step(w.dt, np.eye(3))
    sol = B.from_workload(w, lib=emu)
    st = sol.step(w.dt)
    assert st["newton_chem"] == st_ref["newton_chem"]
    assert rel_err(sol.get(B.FIELD_C), ref.c) < 1e-9
    assert rel_err(sol.get(B.FIELD_F), ref.F) < 1e-8
    sol.close()


def test_emulated_multi_particle_step_matches_oracle(emu):
    """Two particles in one 16^3 periodic RVE, each with its influx band: one coupled step
    against the oracle."""
    w = S.multi_particle(n=16, count=2, rmin=0.15, rmax=0.2, band=2, nsteps=10,
                         phases=S.default_phases(buffer_E=S.BENCH_BUFFER_E))
    prm = oracle_params(w)
    ref = O.CoupledState(prm, w.c_init, w.cdot_B)
    ref.step(w.dt, np.eye(3))
    sol = B.from_workload(w, lib=emu)
    sol.step(w.dt)
    assert rel_err(sol.get(B.FIELD_F), ref.F) < 1e-9
    assert rel_err(sol.get(B.FIELD_C), ref.c) < 1e-10
    sol.close()


def test_emulated_coupled_adjoint_svk_matches_oracle(emu):
    """The coupled adjoint with the Saint-Venant-Kirchhoff law (its tangent and cofactor
    branches of the reverse step) against the oracle's, on the damaging 12 x 12 disc."""
    from oracle import fg_oracle_adjoint as A
    from tests.test_oracle_adjoint import _disc
    shape, logs, src, _, _, phases, pid = _disc(n=12, smax=21e6)
    ph = [O.Phase(law=O.LAW_SVK, E=p.E, nu=p.nu, Omega=p.Omega, c0=p.c0, D=p.D,
                  sigma_max=p.sigma_max) for p in phases]
    prm = O.make_params(ph, pid, (1e-7,) * 3, gc=1.0, lc=2e-7, log_E=logs[0], log_D=logs[2],
                        log_gc=logs[1])
    tols = dict(tol_newton=1e-12, tol_cg=1e-13, tol_chem=1e-12, tol_chem_cg=1e-13,
                tol_pff_cg=1e-13, tol_stag=1e-10, max_stag=400)
    val, g = A.crack_energy_gradient(prm, np.full(shape, 0.01), src, [1.0, 1.0],
                                     [np.eye(3)] * 2, O.Tolerances(**tols))
    assert val > 0.0
    sol = B.Solver(shape, (1e-7,) * 3, ph, pid, src, c_init=np.full(shape, 0.01),
                   log_E=logs[0], log_gc=logs[1], log_D=logs[2], lib=emu, gc=1.0, lc=2e-7,
                   **tols)
    sol.tape(2)
    for _ in range(2):
        sol.step(1.0)
    v2, g2, st = sol.adjoint()
    assert st["gmres"] >= 1
    assert abs(v2 - val) < 1e-8 * val
    for k in ("E", "gc", "D"):
        assert rel_err(g2[k], g[k]) < 1e-9, k
    sol.close()


@pytest.mark.parametrize("shape", [(8, 12, 16), (1, 12, 16), (1, 1, 16)])
@pytest.mark.parametrize("prec", [B.FG_FP64, B.FG_MIXED])
def test_emulated_homogeneous_bar_damages_in_closed_form(emu, shape, prec):
    """Degenerate case of Alg. 4 on 3-D, plane and single-line grids: a homogeneous medium
    without swelling or influx, stretched by F-bar = diag(l, 1, 1) in two steps.  F stays
    F-bar exactly, c is unchanged, no Newton iteration is needed, and the step's single
    staggered pass gives the closed-form H and d (below the threshold at the first
    stretch, damaged at the second)."""
    E, nu, smax, gc, lc = 10e9, 0.3, 50e6, 1.0, 2e-7
    ph = [S.PhaseSpec(E=E, nu=nu, Omega=0.0, c0=0.01, D=1e-14, sigma_max=smax)]
    sol = B.Solver(shape, (1e-7,) * 3, ph, np.zeros(shape, np.uint8), np.zeros(shape),
                   c_init=np.full(shape, 0.2), lib=emu, precision=prec, gc=gc, lc=lc)
    for l, damaged in ((1.002, False), (1.012, True)):
        Fbar = np.diag([l, 1.0, 1.0])
        st = sol.step(1.0, Fbar)
        Hx, dx = homogeneous_stretch_damage(E, nu, smax, gc, lc, l)
        assert (Hx > 0.0) == damaged
        assert st["stag"] == 1 and st["newton_mech"] == 0
        F = sol.get(B.FIELD_F)
        Fx = np.broadcast_to(Fbar.reshape(3, 3, 1, 1, 1), (3, 3) + shape)
        np.testing.assert_allclose(F, Fx, rtol=0, atol=1e-15)
        np.testing.assert_allclose(sol.get(B.FIELD_C), 0.2, rtol=0, atol=1e-15)
        np.testing.assert_allclose(sol.get(B.FIELD_H), Hx, rtol=1e-12)
        np.testing.assert_allclose(sol.get(B.FIELD_D), dx, rtol=1e-9, atol=1e-15)
    sol.close()

def test_emulated_mixed_precision_damage_and_crack_energy(emu):
    """The mixed FP32/FP64 form against the FP64 oracle through three damaging steps of
    the disc with a Gumbel-distributed strength (damage from the first step, d up to 0.93):
    max relative error in F and c <= 1e-7, max |delta d| <= 1e-6 and the fracture energy
    Gamma_E (Eq. crack) of the final d within 1e-6 relative."""
    from tests.test_oracle_adjoint import _strength_disc
    shape, logs, ls, src, prm, phases, pid = _strength_disc()
    ref = O.CoupledState(prm, np.full(shape, 0.01), src, O.Tolerances(max_stag=400))
    sol = B.Solver(shape, (1e-7,) * 3, phases, pid, src, c_init=np.full(shape, 0.01),
                   log_E=logs[0], log_gc=logs[1], log_D=logs[2], log_smax=ls, lib=emu,
                   precision=B.FG_MIXED, gc=1.0, lc=2e-7, max_stag=400)
    for _ in range(3):
        ref.step(1.0, np.eye(3))
        sol.step(1.0)
    d = sol.get(B.FIELD_D)
    assert ref.d.max() > 0.5
    assert rel_err(sol.get(B.FIELD_F), ref.F) <= 1e-7
    assert rel_err(sol.get(B.FIELD_C), ref.c) <= 1e-7
    assert np.abs(d - ref.d).max() <= 1e-6
    g_ref = O.crack_energy(ref.d, prm)
    assert abs(O.crack_energy(d, prm) - g_ref) <= 1e-6 * g_ref
    sol.close()


@pytest.mark.parametrize("shape,prec", [((8, 12, 16), B.FG_FP64), ((1, 12, 16), B.FG_FP64),
                                        ((12, 8, 8), B.FG_MIXED), ((1, 1, 16), B.FG_MIXED)])
def test_emulated_displacement_matches_oracle(emu, shape, prec):
    """Displacement at the voxel corners from F and Fbar (Eq. Fsplit) and its transpose,
    against the oracle, on 3-D, plane and single-line grids of FP64 and mixed contexts
    (the transforms are FP64 in both); also the context's own state."""
    from oracle import fg_oracle_adjoint as A
    rng = np.random.default_rng(5)
    ph = S.default_phases()
    pid = S.random_phase_map(shape, 1)
    h = (1.0e-7, 1.1e-7, 0.9e-7)
    sol = B.Solver(shape, h, ph, pid, np.zeros(shape), lib=emu, precision=prec)
    prm = oracle_params(ph, pid, h)
    F = np.eye(3).reshape(3, 3, 1, 1, 1) + 0.02 * rng.standard_normal((3, 3) + shape)
    Fbar = np.eye(3) + 0.01 * rng.standard_normal((3, 3))
    assert rel_err(sol.displacement(F, Fbar), A.corner_displacement(F, Fbar, prm)) < 1e-13
    r = rng.standard_normal((3,) + shape)
    assert rel_err(sol.displacement_adjoint(r), A.corner_displacement_adjoint(r, prm)) < 1e-13
    np.testing.assert_array_equal(sol.displacement(), 0.0)  # F = Fbar = I initially
    sol.close()


def test_emulated_displacement_mismatch_gradient_matches_oracle(emu):
    """d/dlog(E, g_c, D) of a displacement-mismatch loss after two steps of the disc with a
    Gumbel-distributed strength (damaging from the first step, d up to 0.82), through torch
    autograd (CoupledSteps, then Displacement), against the oracle's adjoint seeded with
    the oracle's dL/dF of the same loss; errors on the common scale of the gradients."""
    import torch
    from oracle import fg_oracle_adjoint as A
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
    geo = B.Solver(shape, w.h, phases, pid, np.zeros(shape), lib=emu)
    t = [torch.tensor(x, requires_grad=True) for x in logs]
    c, F, d = coupled_steps(*t, dict(w=w, nsteps=2, lib=emu, ckpt=1))
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
    # with H = g_c(x)/(2 l_c) D_f the toughness cancels from the phase-field equation, so
    # (c, F, d) and any loss on them do not depend on g_c: that gradient is rounding noise
    assert np.abs(g["gc"]).max() < 1e-12 * scale
    assert np.abs(t[1].grad.numpy()).max() < 1e-12 * scale
    for k, ti in ((("E", t[0]), ("D", t[2]))):
        assert np.abs(ti.grad.numpy() - g[k]).max() < 1e-8 * scale, k
    geo.close()


@pytest.mark.parametrize("law", [S.LAW_NEOHOOKE, S.LAW_SVK])
def test_emulated_krylov_operators_are_symmetric(emu, law):
    """The CUDA operators the conjugate-gradient solves apply are symmetric in FP64,
    independently of the oracle: G K G on compatible fields (made compatible by the
    library's own FP64 projection), the phase-field operator and its preconditioner, and
    the chemistry Newton operator."""
    shape = (8, 12, 16)
    pid = S.random_phase_map(shape, 3)
    phases = S.default_phases(law=law)
    sol = B.Solver(shape, H3, phases, pid, np.zeros(shape), lib=emu)
    F, c, d = S.random_state(shape, seed=6)
    Hh = np.random.default_rng(7).uniform(0, 1e6, shape)
    for f, v in ((B.FIELD_F, F), (B.FIELD_C, c), (B.FIELD_D, d), (B.FIELD_H, Hh)):
        sol.set(f, v)
    rng = np.random.default_rng(9)

    def op(o, v, dt=1.0):
        out = np.zeros_like(v)
        sol.apply(o, np.ascontiguousarray(v), out, 0, dt=dt)
        return out

    def sym(o, a, b, dt=1.0):
        lhs, rhs = float(np.sum(op(o, a, dt) * b)), float(np.sum(a * op(o, b, dt)))
        return abs(lhs - rhs) / max(abs(lhs), abs(rhs))
    x = op(B.OP_GRES, rng.standard_normal((9,) + shape))
    y = op(B.OP_GRES, rng.standard_normal((9,) + shape))
    assert sym(B.OP_MECH, x, y) < 1e-12
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    assert sym(B.OP_PFF, a, b) < 1e-12
    assert sym(B.OP_PFF_PREC, a, b) < 1e-12
    assert sym(B.OP_CHEM, a, b, dt=0.7) < 1e-12
    sol.close()


def test_emulated_damage_does_not_depend_on_the_toughness(emu):
    """The CUDA path keeps the toughness cancellation of the oracle: two damaging steps of
    the 12 x 12 disc with different per-voxel g_c fields give the same (c, F, d) up to the
    solver tolerances and the same H / g_c(x)."""
    from tests.test_oracle_adjoint import _disc
    shape, logs, src, _, _, phases, pid = _disc(n=12, smax=21e6)
    tols = dict(tol_newton=1e-12, tol_stag=1e-10, max_stag=400)
    out = []
    for lg in (logs[1], np.zeros(shape), 0.5 * np.random.default_rng(4).standard_normal(shape)):
        sol = B.Solver(shape, (1e-7,) * 3, phases, pid, src, c_init=np.full(shape, 0.01),
                       log_E=logs[0], log_gc=lg, log_D=logs[2], lib=emu, gc=1.0, lc=2e-7, **tols)
        for _ in range(2):
            sol.step(1.0)
        out.append((sol.get(B.FIELD_C), sol.get(B.FIELD_F), sol.get(B.FIELD_D),
                    sol.get(B.FIELD_H) / np.exp(lg)))
        sol.close()
    assert out[0][2].max() > 0.01
    for o in out[1:]:
        for a, b, t in zip(o, out[0], (1e-14, 1e-12, 1e-9, 1e-9)):
            assert np.abs(a - b).max() <= t * np.abs(b).max()


@pytest.mark.parametrize("ckpt", [1, 2])
def test_emulated_adjoint_under_mixed_control_matches_oracle(emu, ckpt):
    """Reverse pass of two damaging steps with F_xx under stress control (P-bar*_xx = 0):
    the gradient of a seeded loss on the final (c, F, d) against the oracle's adjoint, with
    checkpoints every 1 and 2 steps (F-bar_t from a checkpoint or from mean(F_t))."""
    from oracle import fg_oracle_adjoint as A
    from tests.test_oracle_adjoint import _disc
    shape, logs, src, _, prm_of, phases, pid = _disc(n=12, smax=21e6)
    mask = np.zeros((3, 3), dtype=bool)
    mask[0, 0] = True
    prm = prm_of(*logs)
    prm.stress_mask, prm.Pbar = mask, np.zeros((3, 3))
    tols = dict(tol_newton=1e-12, tol_cg=1e-13, tol_chem=1e-12, tol_chem_cg=1e-13,
                tol_pff_cg=1e-13, tol_stag=1e-10, max_stag=400)
    tol = O.Tolerances(**tols)
    traj = A.forward(prm, np.full(shape, 0.01), src, [1.0, 1.0], [np.eye(3)] * 2, tol)
    rng = np.random.default_rng(12)
    wc, wF, wd = (rng.standard_normal(shape), rng.standard_normal((3, 3) + shape),
                  rng.standard_normal(shape))
    g, _ = A.adjoint(prm, traj, [1.0, 1.0], dict(c=wc, F=wF, d=wd, H=np.zeros(shape)), tol)
    sol = B.Solver(shape, (1e-7,) * 3, phases, pid, src, c_init=np.full(shape, 0.01),
                   log_E=logs[0], log_gc=logs[1], log_D=logs[2], lib=emu, gc=1.0, lc=2e-7,
                   **tols)
    sol.stress_control(mask, np.zeros((3, 3)))
    sol.tape(ckpt)
    for _ in range(2):
        sol.step(1.0)
    assert traj[-1].d.max() > 0.01 and abs(traj[-1].Fbar[0, 0] - 1.0) > 1e-4
    assert rel_err(sol.get(B.FIELD_F), traj[-1].F) < 1e-9
    _, g2, st = sol.adjoint(B.FG_LOSS_SEEDS, seed_c=wc, seed_F=wF, seed_d=wd)
    assert st["steps"] == 2
    scale = max(np.abs(g[k]).max() for k in g)
    for k in ("E", "D"):
        assert np.abs(g2[k] - g[k]).max() < 1e-8 * scale, k
    assert np.abs(g2["gc"]).max() < 1e-12 * scale
    with pytest.raises(B.FgError, match="recorded"):  # one mask for the whole tape
        sol.stress_control(np.zeros((3, 3), dtype=bool), np.zeros((3, 3)))
    sol.close()


@pytest.mark.parametrize("shape", [(8, 12, 16), (1, 100, 100), (12, 8, 8)])
def test_emulated_l2_prefetch_stays_in_bounds_and_changes_nothing(emu, shape):
    """The X passes' L2 prefetch ranges (emulated as reads of each range's first and last
    byte of the bounds-checked buffers) stay inside their buffers on grids with ragged row
    tiles, and the operators and a coupled step give bitwise the same results with and
    without it."""
    out = []
    for pf in (0, 1):
        pid = S.random_phase_map(shape, 1)
        phases = S.default_phases()
        phases[1].E = 2e9
        sol = B.Solver(shape, H3, phases, pid, np.zeros(shape), lib=emu, precision=B.FG_MIXED,
                       l2_prefetch=pf)
        F, c, d = S.random_state(shape, seed=2)
        for f, v in ((B.FIELD_F, F), (B.FIELD_C, c), (B.FIELD_D, d)):
            sol.set(f, v)
        res = []
        x9 = S.random_tensor_field(shape, 3).astype(np.float32)
        x1 = S.random_tensor_field(shape, 4, ncomp=1)[0].astype(np.float32)
        for op, x in ((B.OP_MECH, x9), (B.OP_PFF, x1), (B.OP_CHEM, x1)):
            y = np.zeros_like(x)
            sol.apply(op, x, y, 1)
            res.append(y)
        sol.close()
        w = S.disc2d(n=16, radius=6.0, band=3, nsteps=10)
        s2 = B.from_workload(w, precision=B.FG_MIXED, lib=emu, l2_prefetch=pf)
        s2.step(w.dt)
        res += [s2.get(B.FIELD_F), s2.get(B.FIELD_C)]
        s2.close()
        out.append(res)
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("shape", [(8, 12, 16), (1, 100, 100), (12, 8, 8), (8, 8, 256)])
def test_emulated_float_float_projection_matches_oracle(emu, shape):
    """The float-float residual projection (FG_OP_GRES, prec 2: FP64 fields, transforms in
    pairs of FP32) against the oracle's G * x, element by element, to 1e-13 of the largest
    entry, against 1e-7 for FP32 transforms: it carries the FP64 residual's precision."""
    pid = S.random_phase_map(shape, 1)
    sol = B.Solver(shape, H3, S.default_phases(), pid, np.zeros(shape), lib=emu,
                   precision=B.FG_MIXED)
    x = S.random_tensor_field(shape, 3) * 1e8
    y = np.zeros_like(x)
    sol.apply(B.OP_GRES, x, y, 2)
    ref = O.apply_G(x.reshape((3, 3) + shape), H3)
    assert rel_err(y.reshape(ref.shape), ref) < 1e-13
    y64 = np.zeros_like(x)
    sol.apply(B.OP_GRES, x, y64, 0)
    assert rel_err(y, y64) < 1e-13
    sol.close()




def test_emulated_float_float_residuals_match_fp64_residuals(emu):
    """Mixed-precision steps of the perturbed-particle recipe (16^3) with the residual
    transforms in float-float and in FP64: the same converged fields (both stop at the
    Newton tolerance, so they agree to a few times 1e-10) and the same Krylov counts."""
    import bench
    w = bench._workload(16, 0)
    out = []
    for rff in (1, 0):
        sol = B.from_workload(w, precision=B.FG_MIXED, lib=emu, residual_ff=rff)
        st = [sol.step(w.dt) for _ in range(2)]
        out.append((sol.get(B.FIELD_F), sol.get(B.FIELD_C), st))
        sol.close()
    assert rel_err(out[0][0], out[1][0]) < 1e-9
    assert rel_err(out[0][1], out[1][1]) < 1e-10
    for a, b in zip(out[0][2], out[1][2]):
        assert a["newton_mech"] == b["newton_mech"] and a["newton_chem"] == b["newton_chem"]


@pytest.mark.parametrize("zc", [1, 4])
@pytest.mark.parametrize("shape", [(64, 12, 16), (256, 8, 8), (64, 1, 24)])
def test_emulated_projection_tile_shapes_match_oracle(emu, shape, zc):
    """The FP32 projection pass with 1 and 4 kx-ky columns per block (the autotuner's tile
    shapes) gives the oracle's mechanical operator, ragged last blocks included."""
    pid = S.random_phase_map(shape, 1)
    phases = S.default_phases()
    phases[1].E = 2e9
    sol = B.Solver(shape, H3, phases, pid, np.zeros(shape), lib=emu, precision=B.FG_MIXED,
                   z_columns=zc)
    F, c, d = S.random_state(shape, seed=2)
    for f, v in ((B.FIELD_F, F), (B.FIELD_C, c), (B.FIELD_D, d)):
        sol.set(f, v)
    x = S.random_tensor_field(shape, 3).astype(np.float32)
    y = np.zeros_like(x)
    sol.apply(B.OP_MECH, x, y, 1)
    prm = oracle_params(phases, pid, H3)
    ref = O.mech_apply(F.reshape((3, 3) + shape), c, d, prm, x.astype(float).reshape((3, 3) + shape))
    assert rel_err(y.reshape(ref.shape), ref) < TOL_APPLY_FP32
    sol.close()


@pytest.mark.parametrize("shape", [(128, 128, 8), (128, 128, 12)])
def test_emulated_cluster_yzy_pass_matches_oracle(emu, shape):
    """The clustered Y-Z-Y projection pass (16 CTAs of a cluster per kx plane and tensor row,
    their tiles exchanged through distributed shared memory; emulated one stage of all 16
    CTAs at a time) gives the oracle's mechanical operator, and the three separate passes'
    result to FP32 round-off; also under mixed stress control (the kept zero mode)."""
    pid = S.random_phase_map(shape, 1)
    phases = S.default_phases()
    phases[1].E = 2e9
    F, c, d = S.random_state(shape, seed=2)
    x = S.random_tensor_field(shape, 3).astype(np.float32)
    prm = oracle_params(phases, pid, H3)
    out = {}
    for cp in (1, 0):
        sol = B.Solver(shape, H3, phases, pid, np.zeros(shape), lib=emu, precision=B.FG_MIXED,
                       cluster_pass=cp)
        for f, v in ((B.FIELD_F, F), (B.FIELD_C, c), (B.FIELD_D, d)):
            sol.set(f, v)
        y = np.zeros_like(x)
        sol.apply(B.OP_MECH, x, y, 1)
        mask = np.zeros((3, 3), dtype=bool)
        mask[1, 2] = mask[0, 0] = True
        sol.stress_control(mask, np.zeros((3, 3)))
        ym = np.zeros_like(x)
        sol.apply(B.OP_MECH, x, ym, 1)
        out[cp] = (y, ym)
        sol.close()
    ref = O.mech_apply(F.reshape((3, 3) + shape), c, d, prm, x.astype(float).reshape((3, 3) + shape))
    assert rel_err(out[1][0].reshape(ref.shape), ref) < TOL_APPLY_FP32
    assert rel_err(out[1][0], out[0][0]) < 1e-6
    assert rel_err(out[1][1], out[0][1]) < 1e-6
    assert np.abs(out[1][1] - out[1][0]).max() > 0  # the mask changes the result


@pytest.mark.parametrize("shape", [(128, 128, 8)])
def test_emulated_cluster_chemistry_passes_match_oracle(emu, shape):
    """The chemistry's gradient (1 -> 3) and divergence (3 -> 1) chains as clustered passes:
    the chemistry operator against the oracle's, with the clustered chains and with the
    three-pass chains."""
    pid = S.random_phase_map(shape, 1)
    phases = S.default_phases()
    phases[1].E = 2e9
    F, c, d = S.random_state(shape, seed=2)
    x = S.random_tensor_field(shape, 4, ncomp=1)[0].astype(np.float32)
    prm = oracle_params(phases, pid, H3)
    dt = 0.7
    launches = {}
    for cp in (1, 0):
        sol = B.Solver(shape, H3, phases, pid, np.zeros(shape), lib=emu, precision=B.FG_MIXED,
                       cluster_pass=cp)
        for f, v in ((B.FIELD_F, F), (B.FIELD_C, c), (B.FIELD_D, d)):
            sol.set(f, v)
        y = np.zeros_like(x)
        l0 = B.kernel_launches(emu)
        sol.apply(B.OP_CHEM, x, y, 1, dt=dt)
        launches[cp] = B.kernel_launches(emu) - l0
        Kc = O.chem_conductivity(F.reshape((3, 3) + shape), c, d, prm)
        ref = O.chem_apply(x.astype(float), 1.0 / (c * (1 - c)), Kc, dt, prm)
        assert rel_err(y, ref) < TOL_APPLY_FP32
        sol.close()
    assert launches[1] < launches[0]  # the clustered chains replaced three passes each
