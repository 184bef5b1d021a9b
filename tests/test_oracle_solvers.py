"""Pins of the oracle's solvers (Alg. 1-4) against closed forms, brute force and
invariants that the paper's set-up fixes."""
import math

import numpy as np
import pytest

from oracle import fg_oracle as O
from tests.helpers import homogeneous_stretch_damage

RNG = np.random.default_rng(7)
H = (1e-7, 1e-7, 1e-7)


def two_phase(shape, pid, law=O.LAW_NEOHOOKE, E=(10e9, 2e9), omega=(0.2, 0.0)):
    phases = [O.Phase(law=law, E=E[0], nu=0.3, Omega=omega[0], c0=0.01, D=1e-14),
              O.Phase(law=law, E=E[1], nu=0.25, Omega=omega[1], c0=0.01, D=1e-16)]
    return O.make_params(phases, pid, H, gc=1.0, lc=2e-7)


def identity(shape):
    F = np.zeros((3, 3) + shape)
    for i in range(3):
        F[i, i] = 1.0
    return F


# ---------------------------------------------------------------- mechanics (Alg. 1)

def test_homogeneous_medium_is_uniform_in_one_iteration():
    shape = (4, 4, 4)
    prm = two_phase(shape, np.zeros(shape, dtype=int))
    c = np.full(shape, 0.3)
    d = np.full(shape, 0.2)
    Fbar = np.array([[1.02, 0.01, 0.0], [0.0, 0.99, 0.005], [0.0, 0.0, 1.01]])
    F0 = np.broadcast_to(Fbar.reshape(3, 3, 1, 1, 1), (3, 3) + shape).copy()
    stats = {}
    F, err = O.mech_newton(F0, c, d, prm, Fbar, 1e-9, 1e-10, 5, 100, stats)
    assert err <= 1e-9 and stats.get("newton_mech", 0) == 0
    np.testing.assert_array_equal(F, F0)


@pytest.mark.parametrize("law", [O.LAW_NEOHOOKE, O.LAW_SVK])
def test_laminate_closed_form(law):
    """Phases alternate along x: the exact discrete solution is F = diag(l(x), 1, 1) with
    P_xx equal in both layers and the mean stretch prescribed.  The layer stretches are
    found here by bisection on the scalar uniaxial stress of each law."""
    shape = (2, 3, 8)
    pid = np.zeros(shape, dtype=int)
    pid[:, :, 3:] = 1  # f1 = 3/8, f2 = 5/8
    prm = two_phase(shape, pid, law=law)
    c = np.where(pid == 0, 0.4, 0.01)  # swelling mismatch in layer 1
    d = np.where(pid == 0, 0.1, 0.0)
    Fbar = np.diag([1.01, 1.0, 1.0])

    def pxx(lmb, ph, cc, dd):
        E, nu, om = [(10e9, 0.3, 0.2), (2e9, 0.25, 0.0)][ph]
        lam = E * nu / ((1 + nu) * (1 - 2 * nu))
        mu = E / (2 * (1 + nu))
        a = (1 + om * (cc - 0.01)) ** (-1 / 3)
        le = a * lmb
        if law == O.LAW_NEOHOOKE:
            p0 = mu * (le - 1 / le) + lam * math.log(a ** 3 * lmb) / le
        else:
            exx, eyy = 0.5 * (le * le - 1), 0.5 * (a * a - 1)
            p0 = le * (lam * (exx + 2 * eyy) + 2 * mu * exx)
        return (1 - dd) ** 2 * a * p0

    f1, f2 = 3 / 8, 5 / 8
    g = lambda l1: pxx(l1, 0, 0.4, 0.1) - pxx((1.01 - f1 * l1) / f2, 1, 0.01, 0.0)
    lo, hi = 0.9, 1.1
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(lo) * g(mid) <= 0:
            hi = mid
        else:
            lo = mid
    l1 = 0.5 * (lo + hi)
    l2 = (1.01 - f1 * l1) / f2
    F0 = identity(shape)
    F0[0, 0] = 1.01
    F, err = O.mech_newton(F0, c, d, prm, Fbar, 1e-12, 1e-13, 20, 500)
    ref = np.where(pid == 0, l1, l2)
    np.testing.assert_allclose(F[0, 0], ref, rtol=1e-10)
    np.testing.assert_allclose(F[1, 1], 1.0, atol=1e-12)
    np.testing.assert_allclose(F[2, 2], 1.0, atol=1e-12)
    P = O.stress(F, c, d, prm)
    np.testing.assert_allclose(P[0, 0], P[0, 0].mean(), rtol=1e-9)


def test_cg_matches_dense_solve():
    """Assemble G K G on a 4x4x2 grid column by column and solve it densely (minimum
    norm least squares: the operator is singular on incompatible fields)."""
    shape = (2, 4, 4)
    pid = RNG.integers(0, 2, size=shape)
    prm = two_phase(shape, pid)
    F = identity(shape) + 0.03 * RNG.standard_normal((3, 3) + shape)
    c = RNG.uniform(0.05, 0.5, shape)
    d = RNG.uniform(0.0, 0.4, shape)
    n = 9 * int(np.prod(shape))
    op = lambda x: O.apply_G(O.tangent_apply(F, c, d, prm, O.apply_G(x, H)), H)
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        M[:, k] = op(e.reshape((3, 3) + shape)).ravel()
    assert np.allclose(M, M.T, atol=1e-6 * np.abs(M).max())
    b = -O.apply_G(O.stress(F, c, d, prm), H)
    x_dense = np.linalg.lstsq(M, b.ravel(), rcond=1e-10)[0]
    x_cg, _ = O.cg(lambda x: O.mech_apply(F, c, d, prm, x), b, 1e-13, 2000)
    np.testing.assert_allclose(x_cg.ravel(), x_dense, atol=1e-9 * np.abs(x_dense).max())


# ---------------------------------------------------------------- phase field (Alg. 2)

def pff_params(shape, lc=2e-7, gc=1.0):
    phases = [O.Phase()]
    return O.make_params(phases, np.zeros(shape, dtype=int), H, gc=gc, lc=lc)


def test_pff_uniform_history_closed_form_one_iteration():
    shape = (4, 6, 8)
    prm = pff_params(shape)
    Hh = np.full(shape, 3.7e6)
    stats = {}
    d = O.pff_solve(Hh, np.zeros(shape), prm, 1e-12, 50, stats)
    ref = 2 * 3.7e6 / (prm.gc / prm.lc + 2 * 3.7e6)
    np.testing.assert_allclose(d, ref, rtol=1e-12)
    assert stats["cg_pff"] == 1


def test_pff_1d_crack_discrete_closed_form():
    """History on the plane x = 0 only: off the plane the discrete equation is
    d_{j+1} + d_{j-1} = (2 + h^2/l^2) d_j, so d_j = A (r^j + r^{N-j}) with
    r + 1/r = 2 + h^2/l^2; A follows from the equation on the plane."""
    N = 32
    shape = (1, 2, N)
    lc = 2e-7
    prm = pff_params(shape, lc=lc)
    h = H[0]
    Hh = np.zeros(shape)
    H0 = 5e7
    Hh[..., 0] = H0
    d = O.pff_solve(Hh, np.zeros(shape), prm, 1e-14, 500)
    t = 2 + h * h / (lc * lc)
    r = (t - math.sqrt(t * t - 4)) / 2
    j = np.arange(N)
    prof = r ** j + r ** (N - j)
    # plane equation: (gc/lc + 2H0) d0 - gc lc (d1 - 2 d0 + d_{N-1}) / h^2 = 2 H0
    coef = (prm.gc / prm.lc + 2 * H0) * prof[0] - prm.gc * prm.lc * (prof[1] - 2 * prof[0] + prof[N - 1]) / h ** 2
    A = 2 * H0 / coef
    np.testing.assert_allclose(d[0, 0], A * prof, rtol=1e-10)
    np.testing.assert_allclose(d[0, 1], A * prof, rtol=1e-10)


# ---------------------------------------------------------------- chemistry (Alg. 3)

def shift(u, axis_xyz, s):
    return np.roll(u, -s, axis=-1 - axis_xyz)


def test_chem_operator_is_divergence_stencil():
    """L u = -sum_j [flux_j(x) - flux_j(x - e_j)] / h_j with flux = K grad_f u,
    grad_f the forward difference, for a random symmetric K field."""
    shape = (3, 4, 6)
    h = (0.9e-7, 1.1e-7, 1.0e-7)
    prm = O.make_params([O.Phase()], np.zeros(shape, dtype=int), h, gc=1.0, lc=2e-7)
    A = RNG.standard_normal((3, 3) + shape)
    K = np.einsum("ik...,jk...->ij...", A, A) * 1e-14
    u = RNG.standard_normal(shape)
    g = np.stack([(shift(u, j, 1) - u) / h[j] for j in range(3)])
    flux = np.einsum("jl...,l...->j...", K, g)
    ref = -sum((flux[j] - shift(flux[j], j, -1)) / h[j] for j in range(3))
    np.testing.assert_allclose(O.chem_L(u, K, prm), ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


def _chem_mode_setup(n, amp, kx=1):
    shape = (1, 1, n)
    L = 1.0e-6
    h = (L / n, L / n, L / n)
    phases = [O.Phase(Omega=0.0, D=1e-14)]
    prm = O.make_params(phases, np.zeros(shape, dtype=int), h, gc=1.0, lc=2e-7)
    x = np.arange(n) * h[0]
    k = 2 * np.pi * kx / L
    c_t = 0.3 + amp * np.cos(k * x)
    return prm, c_t.reshape(shape), k, h


def test_chem_single_mode_decay():
    """Small-amplitude Fourier mode, no swelling, F = I, d = 0: each backward-Euler step
    multiplies the amplitude by 1/(1 + 0.9 D dt |xi|^2) (0.9 = phi(0) of Eq. mobility),
    to first order in the amplitude."""
    n, amp = 16, 1e-6
    prm, c_t, k, h = _chem_mode_setup(n, amp)
    F = identity(c_t.shape)
    dt = 0.5
    c = O.chem_solve(c_t, F, np.zeros_like(c_t), dt, np.zeros_like(c_t), prm, 1e-13, 1e-14, 30, 200)
    xi2 = 4 * math.sin(math.pi / n) ** 2 / h[0] ** 2
    fac = 1.0 / (1.0 + 0.9 * 1e-14 * dt * xi2)
    amp_new = 2 * np.abs(np.fft.rfft(c.ravel())[1]) / n
    assert abs(amp_new / amp - fac) < 1e-5
    np.testing.assert_allclose(c.mean(), c_t.mean(), rtol=1e-14)


def _mode_amplitude(c, kx, ky=0):
    """Amplitude a of c = mean + a cos(q . x) from the DFT coefficient of the mode."""
    n_y, n_x = c.shape[-2], c.shape[-1]
    return 2.0 * np.abs(np.fft.fft2(c[0])[ky, kx]) / (n_x * n_y)


def _chem_plane_setup(n, amp, kx, ky, D=1e-14):
    shape = (1, n, n)
    L = 1.0e-6
    h = (L / n, L / n, L / n)
    prm = O.make_params([O.Phase(Omega=0.0, D=D)], np.zeros(shape, dtype=int), h, gc=1.0,
                        lc=2e-7)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    c_t = 0.3 + amp * np.cos(2 * np.pi * (kx * x + ky * y) / n)
    return prm, c_t.reshape(shape), h


@pytest.mark.parametrize("kx,ky", [(1, 0), (0, 1), (1, 2)])
def test_chem_mode_decay_under_shear_follows_inverse_right_cauchy_green(kx, ky):
    """Eq. Jmassflowexpression: the referential mobility carries C^{-1} = (F^T F)^{-1}, the
    pull-back of an isotropic spatial mobility.  Under a uniform simple shear
    F = I + g e_x (x) e_y, a small Fourier mode with forward-difference symbol xi decays per
    backward-Euler step by 1/(1 + 0.9 D dt xi^H C^{-1} xi), C^{-1} = [[1 + g^2, -g], [-g, 1]]
    in the (x, y) block.  The mode along x sees 1 + g^2 (b^{-1} = F^{-T} F^{-1} would give 1,
    C itself 1), the mode along y sees 1 (b^{-1}: 1 + g^2, C: 1 + g^2), the oblique mode
    the off-diagonal -g."""
    n, amp, g, dt = 16, 1e-6, 0.3, 0.5
    prm, c_t, h = _chem_plane_setup(n, amp, kx, ky)
    F = identity(c_t.shape)
    F[0, 1] = g
    c = O.chem_solve(c_t, F, np.zeros_like(c_t), dt, np.zeros_like(c_t), prm, 1e-13, 1e-14,
                     30, 400)
    q = (2 * np.pi * kx / n, 2 * np.pi * ky / n)
    xi = np.array([(np.exp(1j * q[0]) - 1) / h[0], (np.exp(1j * q[1]) - 1) / h[1]])
    Cinv = np.array([[1 + g * g, -g], [-g, 1.0]])
    s = float(np.real(np.conj(xi) @ Cinv @ xi))
    fac = 1.0 / (1.0 + 0.9 * 1e-14 * dt * s)
    assert abs(_mode_amplitude(c, kx, ky) / amp - fac) < 1e-5
    np.testing.assert_allclose(c.mean(), c_t.mean(), rtol=1e-14)


@pytest.mark.parametrize("d0", [0.25, 0.6])
def test_chem_mode_decay_with_uniform_damage_follows_mobility(d0):
    """Eq. mobility: with a uniform phase field d the mobility factor is
    phi(d) = 0.9 (1 - d)^2 + 0.1 d^2, so the mode decays per step by
    1/(1 + phi(d) D dt |xi|^2) (phi(0.25) = 0.5125, phi(0.6) = 0.18)."""
    n, amp, dt = 16, 1e-6, 0.5
    prm, c_t, k, h = _chem_mode_setup(n, amp)
    F = identity(c_t.shape)
    d_t = np.full_like(c_t, d0)
    c = O.chem_solve(c_t, F, d_t, dt, np.zeros_like(c_t), prm, 1e-13, 1e-14, 30, 200)
    phi = {0.25: 0.5125, 0.6: 0.18}[d0]
    xi2 = 4 * math.sin(math.pi / n) ** 2 / h[0] ** 2
    fac = 1.0 / (1.0 + phi * 1e-14 * dt * xi2)
    amp_new = 2 * np.abs(np.fft.rfft(c.ravel())[1]) / n
    assert abs(amp_new / amp - fac) < 1e-5


def test_chem_step_under_shear_equals_isotropic_step_with_scaled_diffusivity():
    """Nonlinear, non-uniform case: for c_t and d_t varying along x only, the x-x entry of
    C^{-1} is the only one the divergence sees, so a step under the simple shear
    F = I + g e_x (x) e_y equals, to solver tolerance, the step at F = I with D (1 + g^2),
    at any concentration profile (Eq. Jmassflowexpression; the whole nonlinear Newton of
    Alg. 3, no linearisation)."""
    n, g, dt = 24, 0.4, 2.0
    shape = (1, 1, n)
    rng = np.random.default_rng(11)
    c_t = rng.uniform(0.05, 0.7, shape)
    d_t = rng.uniform(0.0, 0.8, shape)
    src = np.where(rng.uniform(size=shape) < 0.3, 0.02, 0.0)
    h = (1e-7, 1e-7, 1e-7)
    pid = np.zeros(shape, dtype=int)
    prm = O.make_params([O.Phase(Omega=0.0, D=1e-14)], pid, h, gc=1.0, lc=2e-7)
    prm_iso = O.make_params([O.Phase(Omega=0.0, D=1e-14 * (1 + g * g))], pid, h, gc=1.0,
                            lc=2e-7)
    F = identity(shape)
    F[0, 1] = g
    c_shear = O.chem_solve(c_t, F, d_t, dt, src, prm, 1e-13, 1e-14, 50, 500)
    c_iso = O.chem_solve(c_t, identity(shape), d_t, dt, src, prm_iso, 1e-13, 1e-14, 50, 500)
    assert np.abs(c_shear - c_t).max() > 1e-3  # the step moves c
    np.testing.assert_allclose(c_shear, c_iso, rtol=0, atol=1e-12)


def test_crack_energy_closed_form():
    """Eq. crack, Gamma = sum_voxels g_c (d^2/(2 l_c) + l_c/2 |grad_f d|^2) h_x h_y h_z.  For
    d = d0 + a cos(2 pi k y / n_y) the voxel sums are V (d0^2 + a^2/2) and
    V a^2/2 |xi_y|^2 with |xi_y|^2 = 4 sin^2(pi k / n_y)/h_y^2, so
    Gamma = g_c h_x h_y h_z V [(d0^2 + a^2/2)/(2 l_c) + l_c a^2 |xi_y|^2 / 4]; uniform d (a = 0)
    gives g_c d0^2/(2 l_c) V h_x h_y h_z."""
    shape = (3, 8, 4)
    h = (0.9e-7, 1.1e-7, 1.3e-7)
    lc, gc = 2.5e-7, 1.7
    prm = O.make_params([O.Phase()], np.zeros(shape, dtype=int), h, gc=gc, lc=lc)
    V = np.prod(shape)
    hv = h[0] * h[1] * h[2]
    d0 = 0.3
    np.testing.assert_allclose(O.crack_energy(np.full(shape, d0), prm),
                               gc * d0 * d0 / (2 * lc) * V * hv, rtol=1e-13)
    a, k = 0.2, 3
    y = np.arange(shape[1]).reshape(1, -1, 1)
    d = d0 + a * np.cos(2 * np.pi * k * y / shape[1]) * np.ones(shape)
    xi2 = 4 * math.sin(math.pi * k / shape[1]) ** 2 / h[1] ** 2
    ref = gc * hv * V * ((d0 * d0 + a * a / 2) / (2 * lc) + lc * a * a * xi2 / 4)
    np.testing.assert_allclose(O.crack_energy(d, prm), ref, rtol=1e-12)


def test_chem_mode_converges_to_continuum_decay():
    """Refining h and dt together, the decay approaches exp(-0.9 D k^2 t) (first order
    in dt)."""
    errs = []
    for n, steps in [(16, 4), (32, 8), (64, 16)]:
        prm, c, k, h = _chem_mode_setup(n, 1e-6)
        T = 0.2 / (0.9 * 1e-14 * k * k)
        dt = T / steps
        F = identity(c.shape)
        z = np.zeros_like(c)
        for _ in range(steps):
            c = O.chem_solve(c, F, z, dt, z, prm, 1e-13, 1e-14, 30, 400)
        amp = 2 * np.abs(np.fft.rfft(c.ravel())[1]) / n / 1e-6
        errs.append(abs(amp - math.exp(-0.2)))
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]
    assert errs[2] < 5e-3


def test_chem_mass_balance_with_source():
    shape = (2, 6, 8)
    pid = RNG.integers(0, 2, size=shape)
    phases = [O.Phase(Omega=0.15, D=1e-14), O.Phase(E=1e7, Omega=0.0, D=1e-19)]
    prm = O.make_params(phases, pid, H, gc=1.0, lc=2e-7)
    c_t = RNG.uniform(0.02, 0.3, shape)
    F = identity(shape) + 0.01 * RNG.standard_normal((3, 3) + shape)
    d_t = RNG.uniform(0, 0.3, shape)
    src = np.where(RNG.uniform(size=shape) < 0.3, 0.05, 0.0)
    dt = 1.0
    c = O.chem_solve(c_t, F, d_t, dt, src, prm, 1e-12, 1e-13, 50, 500)
    assert abs(c.mean() - (c_t.mean() + dt * src.mean())) < 1e-12
    Kc = O.chem_conductivity(F, c_t, d_t, prm)
    f = O.chem_residual(c, c_t, F, d_t, Kc, dt, src, prm)
    assert np.abs(f).max() < 1e-10


# ---------------------------------------------------------------- coupled step (Alg. 4)

@pytest.mark.slow
def test_homogeneous_bar_under_stretch_damages_in_closed_form():
    """A homogeneous Neo-Hookean medium (no swelling, no influx) under a macroscopic
    stretch F-bar = diag(l, 1, 1), loaded in two steps of Alg. 4.  The mechanics stays
    uniform, F = F-bar, and each step's body (mechanics, history, phase field) runs once:
    the Cauchy stress is diagonal with sigma_xx = (G (l^2 - 1) + lam ln l)/l and
    sigma_yy = sigma_zz = lam ln l / l, so D_f = sum (<sigma_i>/sigma_max)^2 - 1,
    H = g_c/(2 l_c) D_f (Eq. SigDrivingForce) and, with uniform H, Eq. PFFA gives
    d = 2H/(g_c/l_c + 2H).  The first stretch stays below the threshold (d = 0)."""
    shape = (2, 4, 4)
    E, nu, smax, gc, lc = 10e9, 0.3, 50e6, 1.0, 2e-7
    prm = O.make_params([O.Phase(E=E, nu=nu, Omega=0.0, c0=0.01, sigma_max=smax)],
                        np.zeros(shape, dtype=int), H, gc=gc, lc=lc)
    st = O.CoupledState(prm, np.full(shape, 0.2), np.zeros(shape))
    for l, damaged in ((1.002, False), (1.012, True)):
        Fbar = np.diag([l, 1.0, 1.0])
        stats = st.step(1.0, Fbar)
        Hx, dx = homogeneous_stretch_damage(E, nu, smax, gc, lc, l)
        assert (Hx > 0.0) == damaged
        assert stats["stag"] == 1
        np.testing.assert_allclose(st.F, np.broadcast_to(Fbar.reshape(3, 3, 1, 1, 1),
                                                         (3, 3) + shape), rtol=0, atol=1e-15)
        np.testing.assert_allclose(st.H, Hx, rtol=1e-12)
        np.testing.assert_allclose(st.d, dx, rtol=1e-9, atol=1e-15)
        np.testing.assert_array_equal(st.c, 0.2)


def test_coupled_steps_invariants():
    shape = (1, 16, 16)
    y, x = np.meshgrid(np.arange(16) - 7.5, np.arange(16) - 7.5, indexing="ij")
    part = (x * x + y * y <= 36.0)[None]
    pid = np.where(part, 0, 1)
    phases = [O.Phase(E=10e9, Omega=0.1 / 0.99, D=1e-14, sigma_max=25e6),
              O.Phase(E=10e6, Omega=0.0, D=1e-19, sigma_max=25e6)]
    prm = O.make_params(phases, pid, H, gc=1.0, lc=2e-7)
    src = np.where(part & ~((x * x + y * y) <= 9.0)[None], 0.05, 0.0)
    st = O.CoupledState(prm, np.full(shape, 0.01), src)
    Hprev = st.H.copy()
    for _ in range(3):
        m0 = st.c.mean()
        stats = st.step(1.0, np.eye(3))
        assert abs(st.c.mean() - (m0 + src.mean())) < 1e-11
        assert np.all(st.H >= Hprev)
        assert st.d.min() >= -1e-12 and st.d.max() < 1.0
        _, err = O.mech_residual(st.F, st.c, st.d, prm, np.eye(3))
        assert err <= 1e-9
        Hprev = st.H.copy()
    assert st.H.max() > 0.0  # the band's swelling mismatch reaches the damage threshold


def _cracking_disc():
    shape = (1, 16, 16)
    y, x = np.meshgrid(np.arange(16) - 7.5, np.arange(16) - 7.5, indexing="ij")
    part = (x * x + y * y <= 36.0)[None]
    pid = np.where(part, 0, 1)
    phases = [O.Phase(E=10e9, Omega=0.1 / 0.99, D=1e-14, sigma_max=25e6),
              O.Phase(E=10e6, Omega=0.0, D=1e-19, sigma_max=25e6)]
    prm = O.make_params(phases, pid, H, gc=1.0, lc=2e-7)
    src = np.where(part & ~((x * x + y * y) <= 9.0)[None], 0.05, 0.0)
    return prm, O.CoupledState(prm, np.full(shape, 0.01), src), src


def step_equation_residuals(prm, src, dt, before, after):
    """Residuals of the equations that define one step of Alg. 4, at the state it returned:
    the Fick residual (Eq. Chemresidualfc, relative to |c_t|) with F and d frozen at the
    step's start (Alg. 3; F-bar unchanged, so F at the start is F_t) and K_c from
    (F_t, c_t, d_t); err_res (Eq. mechresiduum) of the final (F, c, d); the history field
    against max(H_t, psi_c D_f(F, c)) (Eq. Hist); the phase-field system of Eq. PFFA with
    that history (relative to |2H|)."""
    F_t, c_t, d_t, H_t = before
    F, c, d, Hf = after
    Kc = O.chem_conductivity(F_t, c_t, d_t, prm)
    f = O.chem_residual(c, c_t, F_t, d_t, Kc, dt, src, prm)
    _, err = O.mech_residual(F, c, d, prm, np.eye(3))
    Hh = O.history_update(H_t, F, c, prm)
    Heff = Hf / O.gc_ratio(prm)
    rd = O.pff_apply(d, Heff, prm) - 2.0 * Heff
    return (np.linalg.norm(f) / np.linalg.norm(c_t), err,
            np.abs(Hf - Hh).max() / max(np.abs(Hh).max(), 1e-300),
            np.linalg.norm(rd) / max(np.linalg.norm(2.0 * Heff), 1e-300))


def test_coupled_step_output_solves_the_step_equations():
    """The state a coupled step returns is the fixed point Alg. 4 defines (the iteration is
    judged by the equations it solves, not by its own stopping tests): three steps of the
    cracking disc, the last with damage, each within the solver tolerances of every
    equation of the step (default tolerances: Newton 1e-9, Krylov 1e-10; the Fick Newton
    stops on |dc| / |c_t| < 1e-9, which leaves a residual below that)."""
    prm, st, src = _cracking_disc()
    for k in range(3):
        before = (st.F.copy(), st.c.copy(), st.d.copy(), st.H.copy())
        st.step(1.0, np.eye(3))
        r_chem, r_mech, r_hist, r_pff = step_equation_residuals(
            prm, src, 1.0, before, (st.F, st.c, st.d, st.H))
        assert r_chem <= 1e-9, (k, r_chem)
        assert r_mech <= 1e-9, (k, r_mech)
        assert r_hist <= 1e-13, (k, r_hist)
        assert r_pff <= 1e-10, (k, r_pff)
    assert st.d.max() > 1e-3  # the last step was checked with damage


def test_cg_truncates_at_nonpositive_curvature():
    """On an indefinite operator CG returns the iterate before the first search direction
    of non-positive curvature: here diag(3, 1, -2) with b = (1, 1, 1), worked by hand.
    x1 = a0 b, a0 = b.b / b.A.b = 3/2; r1 = b - a0 A b = (-7/2, -1/2, 4);
    p1 = r1 + (r1.r1 / b.b) p0 = r1 + (57/2)/3 b = (6, 9, 27/2);
    p1.A.p1 = 108 + 81 - 364.5 < 0  ->  stop with x = x1."""
    A = np.array([3.0, 1.0, -2.0])
    b = np.ones(3)
    stats = {}
    x, it = O.cg(lambda v: A * v, b, 1e-12, 10, stats=stats, indefinite=False)
    np.testing.assert_allclose(x, 1.5 * b, rtol=1e-15)
    assert it == 1 and stats["cg_truncated"] == 1
    with pytest.raises(FloatingPointError):
        O.cg(lambda v: -v, b, 1e-12, 10, indefinite=False)


def test_cg_continues_through_negative_curvature():
    """Taking the direction of negative curvature of the example above, CG reaches the
    exact solution of the 3x3 indefinite system in 3 steps, as it does for any symmetric
    system with 3 distinct eigenvalues while no <p, Ap> vanishes: x = (1/3, 1, -1/2).
    A vanishing <p, Ap> stops it: diag(1, -1) with b = (1, 1) has <b, Ab> = 0."""
    A = np.array([3.0, 1.0, -2.0])
    stats = {}
    x, it = O.cg(lambda v: A * v, np.ones(3), 1e-12, 10, stats=stats)
    np.testing.assert_allclose(x, [1.0 / 3.0, 1.0, -0.5], rtol=1e-13)
    assert it == 3 and stats["cg_negcurv"] >= 1 and "cg_truncated" not in stats
    with pytest.raises(FloatingPointError):
        O.cg(lambda v: np.array([1.0, -1.0]) * v, np.ones(2), 1e-12, 10)


def test_shifted_cg_on_indefinite_system():
    """The shifted re-solve of the mechanical Newton, worked in exact fractions on
    diag(3, 1, -2), b = (1, 1, 1).  Solve 1 (sigma = 0) meets p1 = (6, 9, 27/2) with
    Rayleigh quotient rq = -175.5 / 299.25 = -78/133, so sigma = 2 * 78/133 = 156/133.
    Solve 2 meets p1 = (-2793, 143640, 726579/2) / 134689 with rq = -11307270/26842459, so
    sigma = 2 (156/133 + 11307270/26842459) = 12226188/3834637; A + sigma I is then
    positive definite and solve 3 returns x_i = 1 / (a_i + sigma)."""
    A = np.array([3.0, 1.0, -2.0])
    stats = {}
    x, it, sigma = O.shifted_cg(lambda v: A * v, np.ones(3), 1e-13, 10, stats)
    s_hand = 12226188.0 / 3834637.0
    assert abs(sigma - s_hand) < 1e-13 * s_hand
    np.testing.assert_allclose(x, 1.0 / (A + s_hand), rtol=1e-12)
    assert stats["newton_shifted"] == 2
    # positive definite: no shift, plain CG
    x, it, sigma = O.shifted_cg(lambda v: np.array([3.0, 1.0, 2.0]) * v, np.ones(3), 1e-13, 10)
    assert sigma == 0.0
    np.testing.assert_allclose(x, [1.0 / 3.0, 1.0, 0.5], rtol=1e-12)


def test_minres_solves_indefinite_systems_with_monotone_residual():
    """MINRES on symmetric matrices with eigenvalues of both signs (one of them near zero)
    reaches the dense solution in n steps, and the residual |b - A x_k| of its k-th iterate
    never grows with k, as its minimising property requires."""
    rng = np.random.default_rng(0)
    for n in (6, 10):
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        ev = np.concatenate([rng.uniform(0.5, 3.0, n - 3), [-1.0, -0.2, 0.05]])
        A = Q @ np.diag(ev) @ Q.T
        b = rng.standard_normal(n)
        x, it = O.minres(lambda v: A @ v, b, 1e-13, 100)
        np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
        assert it <= n + 2
        res = [np.linalg.norm(b - A @ O.minres(lambda v: A @ v, b, 0.0, k)[0]) for k in range(1, n + 1)]
        assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(n - 1))
    # a symmetric positive definite system: the same solution as CG
    A = np.diag([3.0, 1.0, 2.0])
    x, _ = O.minres(lambda v: A @ v, np.ones(3), 1e-14, 10)
    np.testing.assert_allclose(x, [1.0 / 3.0, 1.0, 0.5], rtol=1e-13)


def test_cg_truncation_returns_saved_iterate():
    """A truncated solve returns the last iterate saved at a 4x drop of |r|^2 when its own
    residual has grown since: diag(4, 4, 2, -1), b = (1, 1, 1, 1/2), worked by hand.
    |r0|^2 = 13/4, b.A.b = 39/4, a0 = 1/3, x1 = b/3, r1 = (-1, -1, 1, 2)/3, |r1|^2 = 7/9
    <= 13/16 -> saved.  The second step raises |r2|^2 to 40950/361 and the third search
    direction has non-positive curvature, so the solve stops and returns x1.  With maxit = 2
    the cap is reached at the same grown residual and x1 comes back as well."""
    A = np.array([4.0, 4.0, 2.0, -1.0])
    b = np.array([1.0, 1.0, 1.0, 0.5])
    r2 = []

    def op(v):
        return A * v
    stats = {}
    x, it = O.cg(op, b, 1e-12, 10, stats=stats, indefinite=False)
    np.testing.assert_allclose(x, b / 3.0, rtol=1e-15)
    assert it == 2 and stats["cg_truncated"] == 1
    x, it = O.cg(op, b, 1e-12, 2)
    np.testing.assert_allclose(x, b / 3.0, rtol=1e-15)
    # the unguarded second iterate really is worse: its residual is the hand value
    x1 = b / 3.0
    r1 = b - A * x1
    a1 = (r1 @ r1) / ((r1 + (r1 @ r1) / (b @ b) * b) @ (A * (r1 + (r1 @ r1) / (b @ b) * b)))
    r2.append(r1 - a1 * A * (r1 + (r1 @ r1) / (b @ b) * b))
    assert abs(r2[0] @ r2[0] - 40950.0 / 361.0) < 1e-9


def test_mech_adjoint_matches_central_differences():
    """dL/dlogE of L = <W, F(logE)> at equilibrium, against central differences of the
    converged solve on a few voxels."""
    shape = (2, 4, 4)
    rng = np.random.default_rng(3)
    pid = rng.integers(0, 2, size=shape)
    phases = [O.Phase(E=10e9, nu=0.3, Omega=0.2, c0=0.01), O.Phase(E=2e9, nu=0.25, Omega=0.0, c0=0.01)]
    logE = rng.normal(0, 0.1, shape)
    c = rng.uniform(0.05, 0.4, shape)
    d = rng.uniform(0.0, 0.3, shape)
    W = rng.standard_normal((3, 3) + shape)

    def solve(le):
        prm = O.make_params(phases, pid, H, gc=1.0, lc=2e-7, log_E=le)
        F0 = identity(shape)
        F, _ = O.mech_newton(F0, c, d, prm, np.eye(3), 1e-14, 1e-15, 30, 2000)
        return F, prm

    F, prm = solve(logE)
    g = O.mech_adjoint(F, c, d, prm, W, 1e-15, 2000)
    h = 1e-6
    for v in [(0, 0, 0), (1, 2, 3), (0, 3, 1), (1, 1, 2)]:
        lp, lm = logE.copy(), logE.copy()
        lp[v] += h
        lm[v] -= h
        fd = (np.sum(W * solve(lp)[0]) - np.sum(W * solve(lm)[0])) / (2 * h)
        assert abs(fd - g[v]) <= 1e-6 * np.abs(g).max() + 1e-7 * abs(fd)


def test_mixed_control_projection_and_uniaxial_stress():
    """Mixed macroscopic control.  The projection with stress-controlled components M is
    idempotent and self-adjoint and keeps the mean on M only.  A homogeneous Neo-Hookean
    block with F11 = 1.02 prescribed and every other mean stress zero reaches the uniaxial
    state F = diag(1.02, l, l), l found by bisection on P22(diag(1.02, l, l)) = 0 of the
    law itself, and its mean stress vanishes on M."""
    shape = (2, 3, 4)
    phases = [O.Phase(E=10e9, nu=0.3, Omega=0.0, c0=0.01), O.Phase(E=3e9, nu=0.2, Omega=0.0)]
    rng = np.random.default_rng(4)
    prm = O.make_params(phases, (rng.random(shape) < 0.5).astype(int), H, gc=1.0, lc=2e-7)
    mask = np.ones((3, 3), dtype=bool)
    mask[0, 0] = False
    prm.stress_mask, prm.Pbar = mask, np.zeros((3, 3))
    A = rng.standard_normal((3, 3) + shape)
    Bf = rng.standard_normal((3, 3) + shape)
    GA = O.apply_G_mixed(A, prm)
    np.testing.assert_allclose(O.apply_G_mixed(GA, prm), GA, atol=1e-13 * np.abs(GA).max())
    assert abs(O.dot(GA, Bf) - O.dot(A, O.apply_G_mixed(Bf, prm))) < 1e-12 * abs(O.dot(GA, Bf))
    np.testing.assert_allclose(GA.mean(axis=(2, 3, 4)), np.where(mask, A.mean(axis=(2, 3, 4)), 0.0),
                               atol=1e-14)
    hom = O.make_params(phases[:1], np.zeros(shape, dtype=int), H, gc=1.0, lc=2e-7)
    hom.stress_mask, hom.Pbar = mask, np.zeros((3, 3))
    F = identity(shape)
    F[0, 0] = 1.02
    c, d = np.full(shape, 0.01), np.zeros(shape)
    F, err = O.mech_newton(F, c, d, hom, np.diag([1.02, 1.0, 1.0]), 1e-12, 1e-13, 20, 500)
    assert err <= 1e-12

    def p22(l):
        Fe = np.diag([1.02, l, l]).reshape(3, 3, 1, 1, 1)
        one = O.make_params(phases[:1], np.zeros((1, 1, 1), dtype=int), H, gc=1.0, lc=2e-7)
        return O.P0(Fe, one)[1, 1, 0, 0, 0]
    lo, hi = 0.95, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (lo, mid) if p22(lo) * p22(mid) <= 0 else (mid, hi)
    np.testing.assert_allclose(F[:, :, 0, 0, 0], np.diag([1.02, lo, lo]), atol=1e-12)
    P = O.stress(F, c, d, hom).mean(axis=(2, 3, 4))
    assert np.abs(np.where(mask, P, 0.0)).max() < 1e-6 * abs(P[0, 0])


@pytest.mark.parametrize("law", [O.LAW_NEOHOOKE, O.LAW_SVK])
def test_krylov_operators_are_symmetric(law):
    """The operators the conjugate-gradient solves of Algs. 1-3 apply are symmetric:
    G K G on compatible fields (K has major symmetry, G is an orthogonal projection), the
    phase-field operator of Eq. PFFA and its preconditioner (Eq. PFFprecond), and the
    chemistry Newton operator y/m + dt L y (Eq. Chemderfc in y = m dc)."""
    shape = (3, 4, 6)
    pid = RNG.integers(0, 2, size=shape)
    prm = two_phase(shape, pid, law=law)
    rng = np.random.default_rng(41)
    F = identity(shape) + 0.04 * rng.standard_normal((3, 3) + shape)
    c = rng.uniform(0.05, 0.6, shape)
    d = rng.uniform(0.0, 0.5, shape)
    x = O.apply_G(rng.standard_normal((3, 3) + shape), prm.h)
    y = O.apply_G(rng.standard_normal((3, 3) + shape), prm.h)

    def sym(A, a, b):
        lhs, rhs = O.dot(A(a), b), O.dot(a, A(b))
        return abs(lhs - rhs) / max(abs(lhs), abs(rhs))
    assert sym(lambda v: O.mech_apply(F, c, d, prm, v), x, y) < 1e-12
    H = rng.uniform(0.0, 1e6, shape)
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    assert sym(lambda v: O.pff_apply(v, H, prm), a, b) < 1e-12
    assert sym(lambda v: O.pff_precond(v, H.mean(), prm), a, b) < 1e-12
    Kc = O.chem_conductivity(F, c, d, prm)
    assert sym(lambda v: O.chem_apply(v, 1.0 / (c * (1.0 - c)), Kc, 0.7, prm), a, b) < 1e-12
