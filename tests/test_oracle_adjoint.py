"""Pins of the oracle's discrete adjoint (oracle/fg_oracle_adjoint.py) against central
differences of the oracle's own forward functions: every pointwise derivative on random
states of both laws, one reverse step against perturbed steps, and the gradient of the
fracture energy Gamma_E after a short damaging trajectory."""
import numpy as np
import pytest

from oracle import fg_oracle as O
from oracle import fg_oracle_adjoint as A
from paper_2411_16583_gb300 import synth as S

H = (1e-7, 1e-7, 1e-7)
SHAPE = (2, 3, 4)


def _phases(law, smax):
    return [O.Phase(law=law, E=12e9, nu=0.28, Omega=0.2, c0=0.05, D=1e-14, sigma_max=smax),
            O.Phase(law=law, E=3e9, nu=0.33, Omega=0.1, c0=0.05, D=2e-14, sigma_max=smax)]


def _params(law, shape=SHAPE, smax=20e6, seed=0, log_E=None, log_smax=None):
    """Two random phases with a random log g_c field; the same seed gives the same maps."""
    rng = np.random.default_rng(seed)
    pid = (rng.random(shape) < 0.5).astype(int)
    return O.make_params(_phases(law, smax), pid, H, gc=1.3, lc=2e-7, log_E=log_E,
                         log_gc=0.1 * rng.standard_normal(shape), log_smax=log_smax)


def _state(shape=SHAPE, seed=1, amp=0.04):
    rng = np.random.default_rng(seed)
    F = amp * rng.standard_normal((3, 3) + shape)
    for i in range(3):
        F[i, i] += 1.0
    c = rng.uniform(0.1, 0.6, shape)
    d = rng.uniform(0.0, 0.4, shape)
    return F, c, d


def _fd(f, x, dx, h):
    return (f(x + h * dx) - f(x - h * dx)) / (2.0 * h)


@pytest.mark.parametrize("law", [O.LAW_NEOHOOKE, O.LAW_SVK])
def test_stress_and_chemical_potential_derivatives(law):
    prm = _params(law)
    F, c, d = _state()
    h = 1e-6
    np.testing.assert_allclose(A.stress_dc(F, c, d, prm),
                               _fd(lambda x: O.stress(F, x, d, prm), c, 1.0, h), rtol=1e-6,
                               atol=1e-7 * np.abs(O.stress(F, c, d, prm)).max())
    np.testing.assert_allclose(A.stress_dd(F, c, d, prm),
                               _fd(lambda x: O.stress(F, c, x, prm), d, 1.0, h), rtol=1e-6,
                               atol=1e-7 * np.abs(O.stress(F, c, d, prm)).max())
    mue, mue_F, mue_c = A.mu_elastic_derivs(F, c, d, prm)
    np.testing.assert_allclose(mue, O.mu_elastic(F, c, d, prm), rtol=1e-13)
    np.testing.assert_allclose(mue_c, _fd(lambda x: O.mu_elastic(F, x, d, prm), c, 1.0, h),
                               rtol=1e-6, atol=1e-7 * np.abs(mue_c).max())
    dF = np.random.default_rng(5).standard_normal(F.shape)
    np.testing.assert_allclose(O.ddot(mue_F, dF),
                               _fd(lambda x: O.mu_elastic(x, c, d, prm), F, dF, h),
                               rtol=1e-6, atol=1e-7 * np.abs(O.ddot(mue_F, dF)).max())
    # the (1 - d)^2 factor: mu_e(d) = (1 - d)^2 mu_e(0)
    np.testing.assert_allclose(mue, (1.0 - d) ** 2 * O.mu_elastic(F, c, 0.0 * d, prm), rtol=1e-13)


@pytest.mark.parametrize("per_voxel_strength", [False, True])
@pytest.mark.parametrize("law", [O.LAW_NEOHOOKE, O.LAW_SVK])
def test_driving_force_derivatives(law, per_voxel_strength):
    """psi = g_c(x)/(2 l_c) D_f and its derivatives in F, c and log E, on voxels away from
    the Macaulay kink of D_f (the threshold is low enough that most voxels are damaging),
    with a uniform or a per-voxel strength sigma_max(x)."""
    ls = 0.3 * np.random.default_rng(21).standard_normal(SHAPE) if per_voxel_strength else None
    prm = _params(law, smax=60e6, log_smax=ls)
    F, c, _ = _state(amp=0.06)
    psi, Z, psi_c, psi_E = A.psi_terms(F, c, prm)
    np.testing.assert_allclose(psi, prm.gc * O.gc_ratio(prm) / (2 * prm.lc) *
                               O.driving_force(F, c, prm), rtol=1e-13)
    s = O.principal_stresses(O.cauchy_undegraded(F, c, prm))
    t = np.sum((np.maximum(s, 0.0) / prm.sigma_max) ** 2, axis=0)
    safe = np.abs(t - 1.0) > 1e-3
    assert (safe & (t > 1.0)).sum() >= 6 and (safe & (t < 1.0)).sum() >= 2
    h = 1e-7
    dF = np.random.default_rng(6).standard_normal(F.shape)
    fdF = _fd(lambda x: A.psi_terms(x, c, prm)[0], F, dF, h)
    scale = np.abs(psi).max() / np.abs(F).max()
    np.testing.assert_allclose(O.ddot(Z, dF)[safe], fdF[safe], rtol=1e-5, atol=1e-6 * scale)
    fdc = _fd(lambda x: A.psi_terms(F, x, prm)[0], c, 1.0, h)
    np.testing.assert_allclose(psi_c[safe], fdc[safe], rtol=1e-5, atol=1e-6 * np.abs(psi).max())

    def psi_at(logE):
        return A.psi_terms(F, c, _params(law, smax=60e6, log_E=logE, log_smax=ls))[0]
    z = np.zeros(SHAPE)
    fdE = (psi_at(z + h) - psi_at(z - h)) / (2 * h)
    np.testing.assert_allclose(psi_E[safe], fdE[safe], rtol=1e-5, atol=1e-6 * np.abs(psi).max())


def test_conductivity_form_derivative_and_gradient_transpose():
    prm = _params(O.LAW_NEOHOOKE, shape=(3, 4, 5))
    rng = np.random.default_rng(9)
    F, _, _ = _state(shape=(3, 4, 5), amp=0.05)
    c_t = rng.uniform(0.1, 0.6, prm.shape)
    d_t = rng.uniform(0.0, 0.4, prm.shape)
    gl = rng.standard_normal((3,) + prm.shape)
    gm = rng.standard_normal((3,) + prm.shape)

    def s_of(Fx):
        K = O.chem_conductivity(Fx, c_t, d_t, prm)
        return np.einsum("i...,ij...,j...->...", gl, K, gm)
    dF = rng.standard_normal(F.shape)
    got = O.ddot(A.conductivity_form_dF(F, c_t, d_t, gl, gm, prm), dF)
    np.testing.assert_allclose(got, _fd(s_of, F, dF, 1e-6), rtol=1e-6, atol=1e-8 * np.abs(got).max())
    # grad_f^H is the transpose of grad_f: <grad u, f> = <u, grad^H f>
    u = rng.standard_normal(prm.shape)
    f = rng.standard_normal((3,) + prm.shape)
    lhs = O.dot(A.fd_gradient(u, prm), f)
    rhs = O.dot(u, A.fd_divergence_adj(f, prm))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # and grad^H grad is the chemistry operator with K = I
    K = np.zeros((3, 3) + prm.shape)
    for i in range(3):
        K[i, i] = 1.0
    np.testing.assert_allclose(A.fd_divergence_adj(A.fd_gradient(u, prm), prm),
                               O.chem_L(u, K, prm), rtol=1e-10, atol=1e-12 * np.abs(O.chem_L(u, K, prm)).max())


def test_crack_energy_seed():
    prm = _params(O.LAW_NEOHOOKE, shape=(3, 4, 5))
    rng = np.random.default_rng(4)
    d = rng.uniform(0.0, 0.6, prm.shape)
    val, seed, dens = A.crack_energy_seed(d, prm)
    assert abs(val - O.crack_energy(d, prm)) < 1e-13 * val
    assert abs(dens.sum() - val) < 1e-13 * val
    dd = rng.standard_normal(prm.shape)
    fd = _fd(lambda x: O.crack_energy(x, prm), d, dd, 1e-6)
    assert abs(O.dot(seed, dd) - fd) < 1e-7 * abs(fd)
    # direct dependence on log g_c: Gamma is linear in g_c(x), so d/dlog g_c = density
    v = (1, 2, 3)
    up = prm.gcr.copy()
    up[v] *= np.exp(1e-6)
    dn = prm.gcr.copy()
    dn[v] *= np.exp(-1e-6)
    gp = O.crack_energy(d, prm, gc_field=prm.gc * up)
    gm = O.crack_energy(d, prm, gc_field=prm.gc * dn)
    assert abs((gp - gm) / 2e-6 - dens[v]) < 1e-7 * dens[v]


def test_gmres_solves_nonsymmetric_system():
    rng = np.random.default_rng(2)
    M = np.eye(8) + 0.3 * rng.standard_normal((8, 8))
    b = rng.standard_normal(8)
    x, it = A.gmres(lambda v: M @ v, b, 1e-13, 8)
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-10)
    assert it <= 8
    x, it = A.gmres(lambda v: v, np.zeros(8), 1e-13, 8)
    assert it == 0 and not x.any()


# ---------------------------------------------------------------- reverse steps

def _disc(n=10, smax=17e6, seed=3):
    """2D disc particle (radius 0.38 n) in a buffer 100 times softer, influx band of width
    2, per-voxel log E, log g_c, log D ~ N(0, 0.1^2); damage starts in the second step."""
    shape = (1, n, n)
    c0 = (n - 1) / 2
    y, x = np.meshgrid(np.arange(n) - c0, np.arange(n) - c0, indexing="ij")
    R = 0.38 * n
    part = (x * x + y * y <= R * R)[None]
    pid = np.where(part, 0, 1)
    phases = [O.Phase(E=10e9, Omega=0.1 / 0.99, D=1e-14, sigma_max=smax),
              O.Phase(E=1e8, Omega=0.0, D=1e-19, sigma_max=smax)]
    rng = np.random.default_rng(seed)
    logs = [0.1 * rng.standard_normal(shape) for _ in range(3)]
    src = np.where(part & ~((x * x + y * y) <= (R - 2) ** 2)[None], 0.08, 0.0)
    tol = O.Tolerances(tol_newton=1e-13, tol_cg=1e-14, tol_chem=1e-13, tol_chem_cg=1e-14,
                       tol_pff_cg=1e-14, tol_stag=1e-12, max_stag=400)

    def prm_of(lE, lG, lD):
        return O.make_params(phases, pid, H, gc=1.0, lc=2e-7, log_E=lE, log_D=lD, log_gc=lG)
    return shape, logs, src, tol, prm_of, phases, pid


def _strength_disc(n=12, smax=40e6, seed=17):
    """The damaging disc with a per-voxel strength drawn inside the particle with the law
    of Eq. Gumbell (m = 3), as Sec. 5.1 does: its weakest voxel damages in the first step."""
    shape, logs, src, _, _, phases, pid = _disc(n=n, smax=smax)
    ls = np.where(pid == 0, S.gumbel_log_scale(np.random.default_rng(seed), shape), 0.0)
    prm = O.make_params(phases, pid, (1e-7,) * 3, gc=1.0, lc=2e-7, log_E=logs[0], log_D=logs[2],
                        log_gc=logs[1], log_smax=ls)
    return shape, logs, ls, src, prm, phases, pid


@pytest.mark.slow
def test_step_adjoint_matches_central_differences():
    """One reverse step from a damaged state (after two steps) against central differences
    of the third step: a random linear functional of its outputs (c, F, d, H), perturbed
    along random directions of its inputs (c_t, compatible F_t, d_t, H_t) and of the log
    parameters of single voxels.  The history has voxels on both branches of its max."""
    shape, logs, src, tol, prm_of, _, _ = _disc()
    prm = prm_of(*logs)
    traj = A.forward(prm, np.full(shape, 0.01), src, [1.0, 1.0], [np.eye(3)] * 2, tol)
    s_in = traj[-1]
    assert s_in.H.max() > 0.0
    rng = np.random.default_rng(11)
    w = dict(c=rng.standard_normal(shape), F=rng.standard_normal((3, 3) + shape),
             d=rng.standard_normal(shape), H=rng.standard_normal(shape) / s_in.H.max())

    def run(prm_x, c_t, F_t, d_t, H_t):
        st = O.CoupledState(prm_x, c_t, src, tol)
        st.F, st.d, st.H = F_t.copy(), d_t.copy(), H_t.copy()
        st.step(1.0, np.eye(3))
        return st

    def J(st):
        return O.dot(w["c"], st.c) + O.dot(w["F"], st.F) + O.dot(w["d"], st.d) + O.dot(w["H"], st.H)
    out = run(prm, s_in.c, s_in.F, s_in.d, s_in.H)
    psi = A.psi_terms(out.F, out.c, prm)[0]
    assert ((psi > s_in.H) & (s_in.H > 0)).any() or (psi > s_in.H).any()
    assert ((psi < s_in.H) & (s_in.H > 0)).any()
    seeds_in, g = A.step_adjoint(prm, s_in, A.Snapshot(out.c, out.F, out.d, out.H, np.eye(3)),
                                 1.0, w, tol)
    # the staggered loop stops at err_res <= 1e-12, which leaves noise of order 1e-12 / h
    # in a difference quotient: steps of 1e-4 keep it below the truncation error
    h = 1e-4
    dirs = dict(c=0.01 * rng.standard_normal(shape),
                F=O.apply_G(0.01 * rng.standard_normal((3, 3) + shape), prm.h),
                d=0.01 * rng.standard_normal(shape) * (s_in.d > 0),
                H=0.01 * s_in.H.max() * rng.standard_normal(shape) * (s_in.H > 0))
    base = dict(c=s_in.c, F=s_in.F, d=s_in.d, H=s_in.H)
    res = {}
    for k, dv in dirs.items():
        plus = {q: base[q] + (h * dv if q == k else 0) for q in base}
        minus = {q: base[q] - (h * dv if q == k else 0) for q in base}
        fd = (J(run(prm, plus["c"], plus["F"], plus["d"], plus["H"])) -
              J(run(prm, minus["c"], minus["F"], minus["d"], minus["H"]))) / (2 * h)
        res[k] = (O.dot(seeds_in[k], dv), fd)
    scale = max(abs(a) for a, _ in res.values())
    for k, (adj, fd) in res.items():
        assert adj != 0.0 and abs(adj - fd) <= 1e-5 * scale, (k, adj, fd)
    for name, idx in (("E", 0), ("gc", 1), ("D", 2)):
        v = np.unravel_index(np.argmax(np.abs(g[name])), shape)
        lp = [x.copy() for x in logs]
        lm = [x.copy() for x in logs]
        lp[idx][v] += h
        lm[idx][v] -= h
        fd = (J(run(prm_of(*lp), s_in.c, s_in.F, s_in.d, s_in.H)) -
              J(run(prm_of(*lm), s_in.c, s_in.F, s_in.d, s_in.H))) / (2 * h)
        assert abs(g[name][v] - fd) <= 1e-5 * abs(g[name]).max(), (name, g[name][v], fd)


@pytest.mark.slow
def test_crack_energy_gradient_matches_central_differences():
    """dGamma_E/dlog(E, g_c, D) after two steps (damage starts in the second) against
    central differences of the whole forward run, at the voxel of the largest gradient
    of each parameter and at one voxel in the particle's interior."""
    shape, logs, src, tol, prm_of, _, _ = _disc()
    prm = prm_of(*logs)
    stats = {}
    val, g = A.crack_energy_gradient(prm, np.full(shape, 0.01), src, [1.0, 1.0],
                                     [np.eye(3)] * 2, tol, stats)
    assert val > 0.0 and stats["sweeps"] >= 2

    def loss(ls):
        p = prm_of(*ls)
        traj = A.forward(p, np.full(shape, 0.01), src, [1.0, 1.0], [np.eye(3)] * 2, tol)
        return A.crack_energy_seed(traj[-1].d, p)[0]
    h = 1e-6
    for name, idx in (("E", 0), ("gc", 1), ("D", 2)):
        for v in (np.unravel_index(np.argmax(np.abs(g[name])), shape), (0, 5, 5)):
            lp = [x.copy() for x in logs]
            lm = [x.copy() for x in logs]
            lp[idx][v] += h
            lm[idx][v] -= h
            fd = (loss(lp) - loss(lm)) / (2 * h)
            assert abs(g[name][v] - fd) <= 2e-5 * abs(g[name]).max(), (name, v, g[name][v], fd)


# ------------------------------------------------- displacement-mismatch loss (Eq. Fsplit)

def _grid_params(shape, h=(0.7e-7, 1.3e-7, 0.9e-7)):
    return O.make_params([O.Phase()], np.zeros(shape, dtype=int), h, gc=1.0, lc=2e-7)


@pytest.mark.parametrize("shape", [(5, 7, 9), (1, 7, 9), (3, 5, 5)])
def test_corner_displacement_inverts_the_corner_stencil(shape):
    """On odd grids the rotated scheme has no null mode besides k = 0, so a periodic
    corner field u of zero mean, turned into F = Fbar + grad u by the real-space 2x2x2
    stencil, is recovered exactly, together with the affine part (Fbar - I) x."""
    from tests.test_oracle_spectral import corner_gradient
    prm = _grid_params(shape)
    rng = np.random.default_rng(31)
    u = rng.standard_normal((3,) + shape) * 1e-9
    if shape[0] == 1:
        u[2] = 0.0  # plane strain: no out-of-plane displacement
    u -= u.mean(axis=(1, 2, 3), keepdims=True)
    Fbar = np.eye(3) + 0.01 * rng.standard_normal((3, 3))
    if shape[0] == 1:
        Fbar[2, :2] = Fbar[:2, 2] = 0.0
    F = Fbar.reshape(3, 3, 1, 1, 1) + corner_gradient(u, prm.h)
    got = A.corner_displacement(F, Fbar, prm)
    ref = u + np.einsum("ij,j...->i...", Fbar - np.eye(3), A.corner_nodes(prm))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_corner_displacement_on_even_grids_reproduces_compatible_fields():
    """With Nyquist planes the scheme has null modes, which carry no strain: the
    reconstructed u~ then differs from u by them, but its stencil gradient is F - Fbar."""
    from tests.test_oracle_spectral import corner_gradient
    shape = (4, 6, 8)
    prm = _grid_params(shape)
    u = np.random.default_rng(32).standard_normal((3,) + shape) * 1e-9
    F = np.eye(3).reshape(3, 3, 1, 1, 1) + corner_gradient(u, prm.h)
    got = A.corner_displacement(F, np.eye(3), prm)
    np.testing.assert_allclose(corner_gradient(got, prm.h), F - np.eye(3).reshape(3, 3, 1, 1, 1),
                               rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape", [(4, 6, 8), (1, 8, 6), (5, 7, 9)])
def test_corner_displacement_transpose(shape):
    """<u~(F), r> = <F, D^T r> for random F and r (dot-product test of the adjoint map)."""
    prm = _grid_params(shape)
    rng = np.random.default_rng(33)
    F = rng.standard_normal((3, 3) + shape)
    r = rng.standard_normal((3,) + shape)
    lhs = np.sum(A.corner_displacement(F, np.eye(3), prm) * r)
    rhs = np.sum(F * A.corner_displacement_adjoint(r, prm))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.sqrt(np.sum(r * r) * np.sum(F * F)))


def test_displacement_mismatch_seed_is_its_derivative():
    """dL/dF of L = 1/2 sum w |u - u_obs|^2 h^3 against central differences along a
    random direction (L is quadratic in F, so the difference is exact up to rounding)."""
    shape = (3, 4, 6)
    prm = _grid_params(shape)
    rng = np.random.default_rng(34)
    F = np.eye(3).reshape(3, 3, 1, 1, 1) + 0.01 * rng.standard_normal((3, 3) + shape)
    Fbar = np.diag([1.01, 1.0, 0.995])
    u_obs = 1e-9 * rng.standard_normal((3,) + shape)
    w = rng.uniform(0.0, 1.0, shape)
    L, g = A.displacement_mismatch(F, Fbar, u_obs, w, prm)
    dF = rng.standard_normal(F.shape)
    h = 1e-4
    fd = (A.displacement_mismatch(F + h * dF, Fbar, u_obs, w, prm)[0]
          - A.displacement_mismatch(F - h * dF, Fbar, u_obs, w, prm)[0]) / (2 * h)
    assert L > 0.0
    np.testing.assert_allclose(np.sum(g * dF), fd, rtol=1e-8)


def test_damage_does_not_depend_on_the_toughness():
    """With H = g_c(x)/(2 l_c) D_f (Eq. Hist) and the phase-field equation solved divided by
    g_c(x)/g_c, the toughness cancels: two damaging steps with different per-voxel g_c
    fields give the same (c, F, d) up to the solver tolerances, and the same H / g_c(x).
    This is why the toughness gradient of any loss on (c, F, d) vanishes."""
    shape, logs, src, _, prm_of, phases, pid = _disc(n=10, smax=17e6)
    tol = O.Tolerances(tol_newton=1e-12, tol_stag=1e-10, max_stag=400)
    out = []
    for lg in (logs[1], np.zeros(shape), 0.5 * np.random.default_rng(4).standard_normal(shape)):
        st = O.CoupledState(prm_of(logs[0], lg, logs[2]), np.full(shape, 0.01), src, tol)
        for _ in range(2):
            st.step(1.0, np.eye(3))
        out.append((st.c, st.F, st.d, st.H / np.exp(lg)))
    assert out[0][2].max() > 0.01
    for o in out[1:]:
        for a, b, t in zip(o, out[0], (1e-14, 1e-12, 1e-10, 1e-10)):
            assert np.abs(a - b).max() <= t * np.abs(b).max()


@pytest.mark.slow
def test_adjoint_under_mixed_control_matches_central_differences():
    """Two damaging steps with F_xx under stress control (P-bar*_xx = 0, R28): the gradient
    of a random linear loss on the final (c, F, d) against central differences of the whole
    forward run.  Under mixed control the stored Fbar_t is mean(F_t) on the controlled
    component, which the next step's chemistry sees through F~ = F_t + Fcmd - Fbar_t; the
    adjoint that drops this mean dependence misses the E gradient by about 1e-4."""
    shape, logs, src, tol, prm_of, _, _ = _disc(n=10)
    mask = np.zeros((3, 3), dtype=bool)
    mask[0, 0] = True

    def prm_m(*ls):
        p = prm_of(*ls)
        p.stress_mask, p.Pbar = mask, np.zeros((3, 3))
        return p
    rng = np.random.default_rng(12)
    wc, wF, wd = (rng.standard_normal(shape), rng.standard_normal((3, 3) + shape),
                  rng.standard_normal(shape))

    def loss(p):
        traj = A.forward(p, np.full(shape, 0.01), src, [1.0, 1.0], [np.eye(3)] * 2, tol)
        s = traj[-1]
        return float(np.sum(wc * s.c) + np.sum(wF * s.F) + np.sum(wd * s.d)), traj
    L, traj = loss(prm_m(*logs))
    assert traj[-1].d.max() > 0.05 and abs(traj[-1].Fbar[0, 0] - 1.0) > 1e-4
    z = np.zeros(shape)
    g, _ = A.adjoint(prm_m(*logs), traj, [1.0, 1.0], dict(c=wc, F=wF, d=wd, H=z), tol)
    assert np.abs(g["gc"]).max() < 1e-12 * np.abs(g["E"]).max()  # R26: no g_c dependence
    h = 1e-6
    for name, idx, rtol in (("E", 0, 2e-6), ("D", 2, 5e-6)):
        v = np.unravel_index(np.argmax(np.abs(g[name])), shape)
        lp = [x.copy() for x in logs]
        lm = [x.copy() for x in logs]
        lp[idx][v] += h
        lm[idx][v] -= h
        fd = (loss(prm_m(*lp))[0] - loss(prm_m(*lm))[0]) / (2 * h)
        assert abs(g[name][v] - fd) <= rtol * abs(g[name]).max(), (name, v, g[name][v], fd)
