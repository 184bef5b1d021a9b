"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle on the same
seeded inputs.  Operator applications are compared element by element; coupled steps
field by field."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fg_oracle as O
from paper_2411_16583_gb300 import binding as B, synth as S
from tests.helpers import (TOL_APPLY_FF, TOL_APPLY_FP32, TOL_APPLY_FP64, TOL_STEP_FP64,
                           homogeneous_stretch_damage, oracle_params, rel_err)

pytestmark = pytest.mark.gpu

H3 = (1.0e-7, 1.1e-7, 0.9e-7)

# grids spanning several tiles, ragged last tiles (rows not a multiple of the tile) in the
# X, Y and Z passes, mixed radix (12 = 4 x 3, 24 = 8 x 3, 48, 80 = 16 x 5), plane strain
SHAPES = [(8, 12, 16), (12, 24, 16), (1, 12, 16), (1, 64, 64), (16, 32, 64), (24, 48, 80),
          (32, 32, 32), (1, 100, 100), (100, 96, 80),
          # the transform lengths of the 128^3 particle (two-stage 128 = 16 x 8 in every
          # pass) and of the 512^2 disc (512 = 16 x 16 x 2)
          (16, 128, 128), (128, 16, 24), (1, 512, 512), (8, 16, 512),
          # ny = nz = 128: the mixed context's projection chain is the clustered pass
          (128, 128, 16)]


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available()
    return B.load_library()


def _solver(lib, shape, precision, seed=1, law=S.LAW_NEOHOOKE, **kw):
    pid = S.random_phase_map(shape, seed)
    phases = S.default_phases(law=law)
    phases[1].E = 2e9  # moderate contrast keeps the operator well scaled
    sol = B.Solver(shape, H3, phases, pid, np.zeros(shape), lib=lib, precision=precision, **kw)
    F, c, d = S.random_state(shape, seed=seed + 1)
    Hh = np.random.default_rng(seed + 2).uniform(0, 1e6, shape)
    for f, v in ((B.FIELD_F, F), (B.FIELD_C, c), (B.FIELD_D, d), (B.FIELD_H, Hh)):
        sol.set(f, v)
    prm = oracle_params(phases, pid, H3)
    return sol, prm, F.reshape((3, 3) + shape), c, d, Hh


CASES = [(s, S.LAW_NEOHOOKE, 0.0) for s in SHAPES] + [
    ((16, 32, 64), S.LAW_SVK, 0.0),        # the paper's Saint-Venant-Kirchhoff law
    ((32, 32, 32), S.LAW_NEOHOOKE, 1e-5),  # Y-Z-Y passes on many small chunks of kx planes
]


@pytest.mark.parametrize("shape,law,l2f", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_operator_parity(lib, shape, law, l2f, prec):
    sol, prm, F, c, d, Hh = _solver(lib, shape, B.FG_MIXED if prec else B.FG_FP64, law=law,
                                    l2_fraction=l2f)
    tdt = torch.float32 if prec else torch.float64
    tol = TOL_APPLY_FP32 if prec else TOL_APPLY_FP64
    x9 = torch.from_numpy(S.random_tensor_field(shape, 3)).to("cuda", tdt)
    x1 = torch.from_numpy(S.random_tensor_field(shape, 4, ncomp=1)[0]).to("cuda", tdt)
    y9 = torch.empty_like(x9)
    y1 = torch.empty_like(x1)
    xn9 = x9.double().cpu().numpy().reshape(F.shape)
    xn1 = x1.double().cpu().numpy()
    # mechanics  G : F^-1[F[K : x]]
    dot = sol.apply(B.OP_MECH, x9, y9, prec)
    ref = O.mech_apply(F, c, d, prm, xn9)
    assert rel_err(y9.cpu().numpy().reshape(ref.shape), ref) < tol
    assert abs(dot - np.sum(xn9 * ref)) < 10 * tol * np.abs(xn9).sum() * np.abs(ref).max()
    # phase field operator and preconditioner
    sol.apply(B.OP_PFF, x1, y1, prec)
    assert rel_err(y1.cpu().numpy(), O.pff_apply(xn1, Hh, prm)) < tol
    sol.apply(B.OP_PFF_PREC, x1, y1, prec)
    assert rel_err(y1.cpu().numpy(), O.pff_precond(xn1, Hh.mean(), prm)) < tol
    # chemistry Newton operator
    dt = 0.7
    sol.apply(B.OP_CHEM, x1, y1, prec, dt=dt)
    Kc = O.chem_conductivity(F, c, d, prm)
    ref = O.chem_apply(xn1, 1.0 / (c * (1 - c)), Kc, dt, prm)
    assert rel_err(y1.cpu().numpy(), ref) < tol
    if prec == 0:
        sol.apply(B.OP_GRES, x9, y9, 0)
        assert rel_err(y9.cpu().numpy().reshape(F.shape), O.apply_G(xn9, H3)) < tol
    else:  # the residual projection of the mixed mode: FP64 fields, float-float transforms
        x64 = x9.double()
        y64 = torch.empty_like(x64)
        sol.apply(B.OP_GRES, x64, y64, 2)
        assert rel_err(y64.cpu().numpy().reshape(F.shape), O.apply_G(xn9, H3)) < TOL_APPLY_FF
    # stress of the stored state
    assert rel_err(sol.get(B.FIELD_P), O.stress(F, c, d, prm)) < 1e-13
    sol.close()


@pytest.mark.parametrize("prec", [1, 0])
def test_operator_parity_full_size(lib, prec):
    """Every operator at the benchmark size (256^3, where the Y and Z passes take their
    register-direct two-stage form), element by element against the oracle: mechanics,
    phase field and its preconditioner, chemistry, and the residual projection (FP64, and
    float-float in the mixed context)."""
    shape = (256, 256, 256)
    sol, prm, F, c, d, Hh = _solver(lib, shape, B.FG_MIXED if prec else B.FG_FP64, seed=11)
    tdt = torch.float32 if prec else torch.float64
    tol = TOL_APPLY_FP32 if prec else TOL_APPLY_FP64
    x = torch.from_numpy(S.random_tensor_field(shape, 7)).to("cuda", tdt)
    y = torch.empty_like(x)
    xn = x.double().cpu().numpy().reshape(F.shape)
    sol.apply(B.OP_MECH, x, y, prec)
    ref = O.mech_apply(F, c, d, prm, xn)
    assert rel_err(y.cpu().numpy().reshape(ref.shape), ref) < tol
    del ref
    if prec == 0:
        sol.apply(B.OP_GRES, x, y, 0)
        assert rel_err(y.cpu().numpy().reshape(F.shape), O.apply_G(xn, prm.h)) < tol
    else:
        x64 = x.double()
        del y
        y = torch.empty_like(x64)
        sol.apply(B.OP_GRES, x64, y, 2)
        assert rel_err(y.cpu().numpy().reshape(F.shape), O.apply_G(xn, prm.h)) < TOL_APPLY_FF
        del x64
    del x, y, xn
    x1 = torch.from_numpy(S.random_tensor_field(shape, 8, ncomp=1)[0]).to("cuda", tdt)
    y1 = torch.empty_like(x1)
    xn1 = x1.double().cpu().numpy()
    sol.apply(B.OP_PFF, x1, y1, prec)
    assert rel_err(y1.cpu().numpy(), O.pff_apply(xn1, Hh, prm)) < tol
    sol.apply(B.OP_PFF_PREC, x1, y1, prec)
    assert rel_err(y1.cpu().numpy(), O.pff_precond(xn1, Hh.mean(), prm)) < tol
    dt = 0.7
    sol.apply(B.OP_CHEM, x1, y1, prec, dt=dt)
    Kc = O.chem_conductivity(F, c, d, prm)
    ref = O.chem_apply(xn1, 1.0 / (c * (1 - c)), Kc, dt, prm)
    assert rel_err(y1.cpu().numpy(), ref) < tol
    sol.close()


def _oracle_run(w, nsteps):
    prm = oracle_params(w)
    st = O.CoupledState(prm, w.c_init, w.cdot_B, O.Tolerances(**w.tol))
    for _ in range(nsteps):
        st.step(w.dt, np.eye(3))
    return prm, st


def test_coupled_steps_fp64_disc(lib):
    """64 x 64 plane-strain disc (10 steps of influx) in FP64 against the oracle."""
    w = S.disc2d()
    prm, ref = _oracle_run(w, w.nsteps)
    sol = B.from_workload(w, lib=lib)
    for _ in range(w.nsteps):
        st = sol.step(w.dt)
        assert abs(st["mass_err"]) < 1e-12
    assert rel_err(sol.get(B.FIELD_F), ref.F) < TOL_STEP_FP64
    assert rel_err(sol.get(B.FIELD_C), ref.c) < TOL_STEP_FP64
    assert np.abs(sol.get(B.FIELD_D) - ref.d).max() < TOL_STEP_FP64
    sol.close()


def test_coupled_steps_mixed_disc(lib):
    """Mixed FP32/FP64 form on the same disc: per-field error against the oracle."""
    w = S.disc2d()
    nsteps = 4
    prm, ref = _oracle_run(w, nsteps)
    sol = B.from_workload(w, precision=B.FG_MIXED, lib=lib)
    for _ in range(nsteps):
        sol.step(w.dt)
    assert rel_err(sol.get(B.FIELD_F), ref.F) < 1e-7
    assert rel_err(sol.get(B.FIELD_C), ref.c) < 1e-7
    assert np.abs(sol.get(B.FIELD_D) - ref.d).max() < 1e-6
    sol.close()


def test_coupled_step_svk_disc(lib):
    """The paper's Saint-Venant-Kirchhoff law: 3 FP64 steps of the disc against the oracle."""
    w = S.disc2d()
    w.phases = S.default_phases(law=S.LAW_SVK)
    prm, ref = _oracle_run(w, 3)
    sol = B.from_workload(w, lib=lib)
    for _ in range(3):
        sol.step(w.dt)
    assert rel_err(sol.get(B.FIELD_F), ref.F) < TOL_STEP_FP64
    assert rel_err(sol.get(B.FIELD_C), ref.c) < TOL_STEP_FP64
    sol.close()


def test_coupled_step_3d_matches_oracle(lib):
    """A 32^3 rough ellipsoid (the 128^3 particle recipe at a quarter of the size)."""
    w = S.ellipsoid(n=32, axes=(12.5, 10.0, 8.75), rough_std=0.5, rough_corr=1.0, band=2, nsteps=50)
    prm, ref = _oracle_run(w, 1)
    sol = B.from_workload(w, lib=lib)
    sol.step(w.dt)
    assert rel_err(sol.get(B.FIELD_F), ref.F) < TOL_STEP_FP64
    assert rel_err(sol.get(B.FIELD_C), ref.c) < TOL_STEP_FP64
    sol.close()


def test_full_size_step_properties(lib):
    """The 128^3 rough ellipsoid, one FP64 step on the GPU; the oracle then evaluates the
    equilibrium residual and the Fick residual of the GPU's fields, and mass balance."""
    w = S.ellipsoid()
    sol = B.from_workload(w, lib=lib)
    c_t = sol.get(B.FIELD_C)
    F_t = sol.get(B.FIELD_F)
    st = sol.step(w.dt)
    F, c, d = sol.get(B.FIELD_F), sol.get(B.FIELD_C), sol.get(B.FIELD_D)
    prm = oracle_params(w)
    _, err = O.mech_residual(F, c, d, prm, np.eye(3))
    assert err <= 1.5 * w.tol["tol_stag"]
    Kc = O.chem_conductivity(F_t, c_t, np.zeros_like(c), prm)
    f = O.chem_residual(c, c_t, F_t, np.zeros_like(c), Kc, w.dt, w.cdot_B, prm)
    assert np.abs(f).max() < 1e-8
    assert abs(c.mean() - (c_t.mean() + w.dt * w.cdot_B.mean())) < 1e-12
    assert st["stag"] >= 1
    sol.close()


def test_mech_adjoint_autograd_vs_fd_and_oracle(lib):
    """torch.autograd through the hand-written adjoint: dL/dlogE of L = <W, F(logE)>
    against central differences of the GPU forward (h = 1e-6) and the oracle adjoint."""
    from paper_2411_16583_gb300.autograd import mech_equilibrium
    shape = (16, 16, 16)
    rng = np.random.default_rng(21)
    pid = S.random_phase_map(shape, 3)
    phases = S.default_phases()
    phases[1].E = 2e9
    c = rng.uniform(0.05, 0.4, shape)
    d = rng.uniform(0.0, 0.3, shape)
    spec = dict(shape=shape, h=H3, phases=phases, phase_id=pid, c=c, d=d, lib=lib,
                opts=dict(tol_newton=1e-13, tol_cg=1e-14))
    logE = torch.tensor(rng.normal(0, 0.1, shape), dtype=torch.float64, device="cuda",
                        requires_grad=True)
    W = torch.tensor(rng.standard_normal((3, 3) + shape), dtype=torch.float64, device="cuda")
    F = mech_equilibrium(logE, spec)
    (W * F).sum().backward()
    g = logE.grad.cpu().numpy()
    prm = O.make_params([O.Phase(**vars(p)) for p in phases], pid, H3, gc=1.0, lc=2e-7,
                        log_E=logE.detach().cpu().numpy())
    ref = O.mech_adjoint(F.detach().cpu().numpy(), c, d, prm, W.cpu().numpy(), 1e-14, 3000)
    assert rel_err(g, ref) < 1e-6
    h = 1e-6
    for v in [(0, 0, 0), (5, 9, 3), (15, 2, 11), (8, 8, 8)]:
        lp, lm = logE.detach().clone(), logE.detach().clone()
        lp[v] += h
        lm[v] -= h
        fd = ((W * mech_equilibrium(lp, spec)).sum() - (W * mech_equilibrium(lm, spec)).sum()).item() / (2 * h)
        # the forward solves converge to err_res 1e-13: differences at h = 1e-6 carry
        # noise of about 1e-6 of the largest gradient entry
        assert abs(fd - g[v]) <= 1e-5 * np.abs(g).max()


def test_batch_members_equal_solo_runs(lib):
    """Uneven RVEs (48^3 to 96^3 spheres) stepped as one batch on concurrent streams give
    the same fields as each RVE stepped alone."""
    ws = [S.sphere(n, r, band=3, nsteps=20, seed=i)
          for i, (n, r) in enumerate([(48, 0.3), (64, 0.4), (80, 0.35), (96, 0.45)])]
    solo = [B.from_workload(w, precision=B.FG_MIXED, lib=lib) for w in ws]
    for s_, w in zip(solo, ws):
        s_.step(w.dt)
    members = [B.from_workload(w, precision=B.FG_MIXED, lib=lib) for w in ws]
    for m in members:
        m.autotune()
    batch = B.Batch(members)
    stats = batch.step(1.0)
    assert all(st["status"] == 0 for st in stats)
    for a, b in zip(members, solo):
        assert rel_err(a.get(B.FIELD_F), b.get(B.FIELD_F)) < 1e-12
        assert rel_err(a.get(B.FIELD_C), b.get(B.FIELD_C)) < 1e-12
    batch.close()
    for s_ in solo + members:
        s_.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_grouped_batch_apply_equals_member_applies(lib, prec):
    """Grouped launches over a batch (one launch per pass over every member of a grid, the
    members' pass arguments in a device table): six spheres of 48^3, 64^3 and 96^3 give, bit
    for bit, each member's own fg_apply; the oracle's operator checks one member; the
    timing entry point runs all four schedules."""
    ws = [S.sphere(n, r, band=3, nsteps=20, seed=i)
          for i, (n, r) in enumerate([(48, 0.3), (64, 0.4), (48, 0.35), (96, 0.45), (64, 0.3),
                                      (48, 0.4)])]
    members = [B.from_workload(w, precision=B.FG_MIXED, lib=lib) for w in ws]
    gen = torch.Generator(device="cuda").manual_seed(5)
    dt = torch.float32 if prec == 1 else torch.float64
    xs = [torch.randn((9,) + w.shape, generator=gen, device="cuda", dtype=dt) for w in ws]
    solo = []
    for m, x in zip(members, xs):
        y = torch.zeros_like(x)
        m.apply(B.OP_MECH, x, y, prec)
        solo.append(y)
    batch = B.Batch(members)
    ys = [torch.zeros_like(x) for x in xs]
    batch.apply(xs, ys, prec)
    torch.cuda.synchronize()
    for y, ref in zip(ys, solo):
        assert torch.equal(y, ref)
    w = ws[1]
    prm = oracle_params(w)
    F = members[1].get(B.FIELD_F).reshape((3, 3) + w.shape)
    ref = O.mech_apply(F, members[1].get(B.FIELD_C), members[1].get(B.FIELD_D), prm,
                       xs[1].double().cpu().numpy().reshape((3, 3) + w.shape))
    tol = TOL_APPLY_FP32 if prec == 1 else TOL_APPLY_FP64
    assert rel_err(ys[1].double().cpu().numpy().reshape(ref.shape), ref) < tol
    ms, info = batch.time_apply(prec=prec, n=3)
    assert info[0] == 3 and info[1] < info[2] and all(t > 0 for t in ms)
    batch.close()
    for m in members:
        m.close()


def test_mixed_vs_fp64_gpu_perturbed_particle(lib):
    """The perturbed-particle recipe of the 256^3 benchmark at 64^3: three coupled steps
    in the mixed form against the FP64 GPU form at Newton tolerance 1e-9."""
    import bench
    w = bench._workload(64, 0)
    a = B.from_workload(w, lib=lib)
    b = B.from_workload(w, precision=B.FG_MIXED, lib=lib)
    for _ in range(3):
        a.step(w.dt)
        b.step(w.dt)
    assert rel_err(b.get(B.FIELD_F), a.get(B.FIELD_F)) < 1e-7
    assert rel_err(b.get(B.FIELD_C), a.get(B.FIELD_C)) < 1e-7
    assert np.abs(b.get(B.FIELD_D) - a.get(B.FIELD_D)).max() < 1e-6
    a.close()
    b.close()


def test_per_voxel_strength_matches_oracle(lib):
    """Per-voxel strength sigma_max(x) drawn with the law of Eq. Gumbell (Sec. 5.1), with
    per-voxel log E, log D and log g_c: two FP64 steps on the device, damaging from the
    first, against the oracle (F, c, H, d)."""
    from tests.test_oracle_adjoint import _strength_disc
    shape, logs, ls, src, prm, phases, pid = _strength_disc()
    tols = dict(tol_newton=1e-12, tol_stag=1e-10, max_stag=400)
    ref = O.CoupledState(prm, np.full(shape, 0.01), src, O.Tolerances(**tols))
    sol = B.Solver(shape, (1e-7,) * 3, phases, pid, src, c_init=np.full(shape, 0.01),
                   log_E=logs[0], log_gc=logs[1], log_D=logs[2], log_smax=ls, lib=lib, gc=1.0,
                   lc=2e-7, **tols)
    for _ in range(2):
        ref.step(1.0, np.eye(3))
        sol.step(1.0)
    assert ref.d.max() > 0.5
    assert rel_err(sol.get(B.FIELD_F), ref.F) < 1e-8
    assert rel_err(sol.get(B.FIELD_C), ref.c) < 1e-8
    assert rel_err(sol.get(B.FIELD_H), ref.H) < 1e-8
    assert np.abs(sol.get(B.FIELD_D) - ref.d).max() < 1e-8
    sol.close()


def test_gumbel_svk_disc_step(lib):
    """The paper's 2D example type (Sec. 5.1): a 512^2 Saint-Venant-Kirchhoff disc with
    Weibull-distributed stiffness and strength; two mixed steps, the second one damaging
    at the weakest voxels, then the oracle's residuals of the GPU's fields."""
    w = S.gumbel_disc()
    sol = B.from_workload(w, precision=B.FG_MIXED, lib=lib)
    for _ in range(2):
        st = sol.step(w.dt)
        assert st["status"] == 0
    F, c, d = sol.get(B.FIELD_F), sol.get(B.FIELD_C), sol.get(B.FIELD_D)
    assert st["stag"] > 1 and d.max() > 1e-3
    prm = oracle_params(w)
    _, err = O.mech_residual(F, c, d, prm, np.eye(3))
    assert err <= 2 * w.tol["tol_stag"]
    sol.close()


ADJ_TOLS = dict(tol_newton=1e-12, tol_cg=1e-13, tol_chem=1e-12, tol_chem_cg=1e-13,
                tol_pff_cg=1e-13, tol_stag=1e-10, max_stag=400)


@pytest.mark.parametrize("ckpt", [1, 2])
def test_coupled_adjoint_matches_oracle(lib, ckpt):
    """dGamma_E/dlog(E, g_c, D) on the GPU (tape, recompute from checkpoints, transposed
    block sweeps with GMRES, chemistry transpose, FP64) against the oracle's adjoint, on
    two steps of a 12 x 12 disc whose second step damages."""
    from oracle import fg_oracle_adjoint as A
    from tests.test_oracle_adjoint import _disc
    shape, logs, src, _, prm_of, phases, pid = _disc(n=12, smax=21e6)
    prm = prm_of(*logs)
    val, g = A.crack_energy_gradient(prm, np.full(shape, 0.01), src, [1.0, 1.0],
                                     [np.eye(3)] * 2, O.Tolerances(**ADJ_TOLS))
    sol = B.Solver(shape, (1e-7,) * 3, phases, pid, src, c_init=np.full(shape, 0.01),
                   log_E=logs[0], log_gc=logs[1], log_D=logs[2], lib=lib, gc=1.0, lc=2e-7,
                   **ADJ_TOLS)
    sol.tape(ckpt)
    for _ in range(2):
        sol.step(1.0)
    d_before = sol.get(B.FIELD_D)
    v2, g2, st = sol.adjoint()
    assert st["steps"] == 2 and st["recomputed"] == 2 and st["gmres"] >= 1
    assert abs(v2 - val) < 1e-8 * val
    for k in ("E", "gc", "D"):
        assert rel_err(g2[k], g[k]) < 1e-9, k
    np.testing.assert_array_equal(sol.get(B.FIELD_D), d_before)
    # the same gradients through FG_LOSS_SEEDS with the crack energy's seed dGamma/dd
    _, seed_d, dens = A.crack_energy_seed(d_before, prm)
    _, gs, _ = sol.adjoint(B.FG_LOSS_SEEDS, seed_d=seed_d)
    assert rel_err(gs["E"], g2["E"]) < 1e-9 and rel_err(gs["D"], g2["D"]) < 1e-9
    assert rel_err(gs["gc"] + dens, g2["gc"]) < 1e-9
    sol.close()


def test_coupled_adjoint_3d_checkpoint_spacing(lib):
    """A 32^3 sphere with log fields, four FP64 steps at the default tolerances, a loss with
    random seeds on the final (c, F, d): the gradients do not depend on the checkpoint
    spacing (1, 2 or 4 steps per segment: the recomputed steps repeat the recorded ones),
    and the stored state is the one before the call."""
    w = S.with_log_fields(S.sphere(32, 0.35, band=3, nsteps=8,
                                   phases=S.default_phases(buffer_E=S.BENCH_BUFFER_E)), std=0.1)
    rng = np.random.default_rng(5)
    seeds = dict(seed_c=rng.standard_normal(w.shape), seed_F=rng.standard_normal((3, 3) + w.shape),
                 seed_d=rng.standard_normal(w.shape))
    out = {}
    for ckpt in (1, 2, 4):
        sol = B.from_workload(w, lib=lib)
        sol.tape(ckpt)
        for _ in range(4):
            sol.step(w.dt)
        F0 = sol.get(B.FIELD_F)
        out[ckpt] = sol.adjoint(B.FG_LOSS_SEEDS, **seeds)
        np.testing.assert_array_equal(sol.get(B.FIELD_F), F0)
        sol.close()
    # no damage in four steps: g_c cannot act and its gradient is exactly zero
    assert np.abs(out[1][1]["E"]).max() > 0.0 and np.abs(out[1][1]["D"]).max() > 0.0
    for k in ("E", "gc", "D"):
        for ckpt in (2, 4):
            assert rel_err(out[ckpt][1][k], out[1][1][k]) < 1e-9, (ckpt, k)
    assert out[4][2]["recomputed"] == 4 and out[1][2]["steps"] == 4


def test_mixed_control_step_matches_oracle(lib):
    """Two coupled FP64 steps of a swelling disc under mixed macroscopic control (F11
    prescribed, every other mean stress zero) against the oracle, including the solved
    mean deformation gradient."""
    w = S.disc2d(n=32, radius=11.0, band=3, nsteps=10)
    prm = oracle_params(w)
    mask = np.ones((3, 3), dtype=bool)
    mask[0, 0] = False
    prm.stress_mask, prm.Pbar = mask, np.zeros((3, 3))
    tols = dict(tol_newton=1e-12, tol_cg=1e-13, tol_stag=1e-11)
    ref = O.CoupledState(prm, w.c_init, w.cdot_B, O.Tolerances(**tols))
    sol = B.from_workload(w, lib=lib, **tols)
    sol.stress_control(mask, np.zeros((3, 3)))
    for k in range(2):
        Fbar = np.diag([1.0 + 0.005 * (k + 1), 1.0, 1.0])
        ref.step(w.dt, Fbar)
        sol.step(w.dt, Fbar)
    F = sol.get(B.FIELD_F)
    assert rel_err(F, ref.F) < 1e-9
    assert rel_err(sol.get(B.FIELD_C), ref.c) < 1e-10
    np.testing.assert_allclose(F.mean(axis=(2, 3, 4)), ref.Fbar, atol=1e-12)
    sol.close()


def test_cg_graph_replay_is_bitwise_identical(lib):
    """The mechanical CG replays chunks of 16 iterations from captured CUDA graphs on streams
    that can be captured: two steps of the 64^3 benchmark recipe on a side stream equal, bit
    for bit, the same steps on the legacy default stream (where nothing is captured)."""
    import bench
    w = bench._workload(64, 0)
    side = torch.cuda.Stream()
    a = B.from_workload(w, precision=B.FG_MIXED, stream=side.cuda_stream, lib=lib)
    b = B.from_workload(w, precision=B.FG_MIXED, lib=lib)
    replays = 0
    for _ in range(2):
        sa = a.step(w.dt)
        sb = b.step(w.dt)
        assert sa["cg_mech"] == sb["cg_mech"] and sa["cg_mech"] > 48
        assert sb["cg_graph_replays"] == 0
        replays += sa["cg_graph_replays"]
    assert replays > 0
    for f in (B.FIELD_F, B.FIELD_C, B.FIELD_D):
        np.testing.assert_array_equal(a.get(f), b.get(f))
    a.close()
    b.close()


def test_coupled_steps_autograd_gpu(lib):
    """torch autograd through CoupledSteps on the GPU: a directional derivative of a loss on
    the final (c, F, d) agrees with central differences of the forward (damaging disc)."""
    from paper_2411_16583_gb300.autograd import coupled_steps
    from tests.test_oracle_adjoint import _disc
    shape, logs, src, _, _, phases, pid = _disc(n=12, smax=21e6)
    w = S.Workload(name="disc12", shape=shape, h=(1e-7,) * 3, phases=phases,
                   phase_id=pid.astype(np.uint8), cdot_B=src, c_init=np.full(shape, 0.01),
                   gc=1.0, lc=2e-7, dt=1.0, nsteps=2)
    w.tol = dict(ADJ_TOLS)
    spec = dict(w=w, nsteps=2, lib=lib, ckpt=1)
    rng = np.random.default_rng(1)
    wc, wd = rng.standard_normal(shape), rng.standard_normal(shape)
    wF = rng.standard_normal((3, 3) + shape)

    def loss_of(lE, lG, lD):
        c, F, d = coupled_steps(lE, lG, lD, spec)
        return ((c * torch.from_numpy(wc)).sum() + (F * torch.from_numpy(wF)).sum()
                + (d * torch.from_numpy(wd)).sum())
    t = [torch.tensor(x, requires_grad=True) for x in logs]
    loss_of(*t).backward()
    h = 1e-4
    dirs = [0.3 * rng.standard_normal(shape) for _ in range(3)]
    with torch.no_grad():
        lp = loss_of(*[torch.tensor(x + h * dx) for x, dx in zip(logs, dirs)]).item()
        lm = loss_of(*[torch.tensor(x - h * dx) for x, dx in zip(logs, dirs)]).item()
    fd = (lp - lm) / (2 * h)
    adj = sum(float((ti.grad.numpy() * dx).sum()) for ti, dx in zip(t, dirs))
    assert abs(adj - fd) <= 1e-5 * abs(fd), (adj, fd)


@pytest.mark.parametrize("shape", [(32, 48, 64), (1, 64, 64)])
@pytest.mark.parametrize("prec", [B.FG_FP64, B.FG_MIXED])
def test_homogeneous_bar_damages_in_closed_form(lib, shape, prec):
    """Degenerate case of Alg. 4 on the device: a homogeneous medium without swelling or
    influx, stretched by F-bar = diag(l, 1, 1) in two steps, keeps F = F-bar and c, needs
    no Newton iteration, and its single staggered pass gives the closed-form H and d
    (undamaged at the first stretch, damaged at the second)."""
    E, nu, smax, gc, lc = 10e9, 0.3, 50e6, 1.0, 2e-7
    ph = [S.PhaseSpec(E=E, nu=nu, Omega=0.0, c0=0.01, D=1e-14, sigma_max=smax)]
    sol = B.Solver(shape, (1e-7,) * 3, ph, np.zeros(shape, np.uint8), np.zeros(shape),
                   c_init=np.full(shape, 0.2), lib=lib, precision=prec, gc=gc, lc=lc)
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

def test_mixed_precision_damage_and_crack_energy(lib):
    """The mixed FP32/FP64 form against the FP64 oracle through three damaging steps of
    the disc with a Gumbel-distributed strength (damage from the first step, d up to 0.93):
    max relative error in F and c <= 1e-7, max |delta d| <= 1e-6 and the fracture energy
    Gamma_E (Eq. crack) of the final d within 1e-6 relative."""
    from tests.test_oracle_adjoint import _strength_disc
    shape, logs, ls, src, prm, phases, pid = _strength_disc()
    ref = O.CoupledState(prm, np.full(shape, 0.01), src, O.Tolerances(max_stag=400))
    sol = B.Solver(shape, (1e-7,) * 3, phases, pid, src, c_init=np.full(shape, 0.01),
                   log_E=logs[0], log_gc=logs[1], log_D=logs[2], log_smax=ls, lib=lib,
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


def test_float_float_residuals_match_fp64_residuals(lib):
    """The mixed form with its residual transforms in float-float and in FP64, three steps
    of the 64^3 perturbed-particle recipe from the same start: the same Newton iterations
    and fields that agree to the solver tolerance."""
    import bench
    w = bench._workload(64, 0)
    out = []
    for rff in (1, 0):
        sol = B.from_workload(w, precision=B.FG_MIXED, lib=lib, residual_ff=rff)
        st = [sol.step(w.dt) for _ in range(3)]
        out.append((sol.get(B.FIELD_F), sol.get(B.FIELD_C), st))
        sol.close()
    assert rel_err(out[0][0], out[1][0]) < 1e-9
    assert rel_err(out[0][1], out[1][1]) < 1e-10
    for a, b in zip(out[0][2], out[1][2]):
        assert a["newton_mech"] == b["newton_mech"] and a["newton_chem"] == b["newton_chem"]
