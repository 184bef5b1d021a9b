"""Pins of the oracle's constitutive law, chemical potential and damage driving force
(Sec. 2.1, Eqs. Fc, Ee, psie0, psiedamaged, Pderivada, SigDrivingForce; Sec. 2.2 Eq. mue).
"""
import numpy as np
import pytest

from oracle import fg_oracle as O

RNG = np.random.default_rng(99)
SHAPE = (2, 3, 4)


def params(law, omega=0.2, c0=0.01):
    phases = [O.Phase(law=law, E=12e9, nu=0.28, Omega=omega, c0=c0, sigma_max=80e6),
              O.Phase(law=law, E=3e9, nu=0.35, Omega=0.0, c0=c0, sigma_max=80e6)]
    pid = RNG.integers(0, 2, size=SHAPE)
    return O.make_params(phases, pid, (1e-7, 1e-7, 1e-7), gc=1.0, lc=2e-7)


def rand_state(amp=0.05):
    F = np.eye(3).reshape(3, 3, 1, 1, 1) + amp * RNG.standard_normal((3, 3) + SHAPE)
    c = RNG.uniform(0.05, 0.6, SHAPE)
    d = RNG.uniform(0.0, 0.6, SHAPE)
    return F, c, d


LAWS = [O.LAW_NEOHOOKE, O.LAW_SVK]


@pytest.mark.parametrize("law", LAWS)
def test_stress_is_energy_derivative(law):
    prm = params(law)
    F, c, d = rand_state()
    P = O.stress(F, c, d, prm)
    eps = 1e-6
    for i in range(3):
        for j in range(3):
            Fp, Fm = F.copy(), F.copy()
            Fp[i, j] += eps
            Fm[i, j] -= eps
            fd = (O.psi_e(Fp, c, d, prm) - O.psi_e(Fm, c, d, prm)) / (2 * eps)
            np.testing.assert_allclose(P[i, j], fd, rtol=1e-6, atol=1e-8 * np.abs(P).max())


@pytest.mark.parametrize("law", LAWS)
def test_tangent_is_stress_derivative_and_symmetric(law):
    prm = params(law)
    F, c, d = rand_state()
    A = RNG.standard_normal((3, 3) + SHAPE)
    B = RNG.standard_normal((3, 3) + SHAPE)
    eps = 1e-6
    fd = (O.stress(F + eps * A, c, d, prm) - O.stress(F - eps * A, c, d, prm)) / (2 * eps)
    KA = O.tangent_apply(F, c, d, prm, A)
    np.testing.assert_allclose(KA, fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())
    KB = O.tangent_apply(F, c, d, prm, B)
    np.testing.assert_allclose(O.ddot(A, KB), O.ddot(B, KA), rtol=1e-10)


@pytest.mark.parametrize("law", LAWS)
def test_small_strain_limit_is_linear_elasticity(law):
    """For F = I + e with |e| -> 0 at c = c0, d = 0: P = lam tr(e) I + 2 G sym(e)."""
    prm = params(law)
    c = np.full(SHAPE, 0.01)
    d = np.zeros(SHAPE)
    e = 1e-7 * RNG.standard_normal((3, 3) + SHAPE)
    F = np.eye(3).reshape(3, 3, 1, 1, 1) + e
    P = O.stress(F, c, d, prm)
    lam, mu = prm.lam, prm.mu
    tr = e[0, 0] + e[1, 1] + e[2, 2]
    ref = 2 * mu * 0.5 * (e + np.swapaxes(e, 0, 1))
    for i in range(3):
        ref[i, i] += lam * tr
    np.testing.assert_allclose(P, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


@pytest.mark.parametrize("law", LAWS)
def test_free_swelling_and_degradation(law):
    prm = params(law)
    c = RNG.uniform(0.05, 0.6, SHAPE)
    d = RNG.uniform(0.0, 0.9, SHAPE)
    # stress free at the reference concentration
    I = np.broadcast_to(np.eye(3).reshape(3, 3, 1, 1, 1), (3, 3) + SHAPE).copy()
    np.testing.assert_allclose(O.stress(I, prm.c0, d, prm), 0.0, atol=1e-3)
    # free isotropic swelling F = J_c^{1/3} I, J_c = 1 + Omega (c - c0), is stress free
    Jc = 1.0 + prm.Omega * (c - prm.c0)
    Fs = I * Jc ** (1.0 / 3.0)
    np.testing.assert_allclose(O.stress(Fs, c, d, prm), 0.0, atol=1e-3)
    # degradation (1-d)^2
    F, _, _ = rand_state()
    np.testing.assert_allclose(O.stress(F, c, d, prm), (1 - d) ** 2 * O.stress(F, c, 0 * d, prm),
                               rtol=1e-12)


@pytest.mark.parametrize("law", LAWS)
def test_objectivity(law):
    prm = params(law)
    F, c, d = rand_state()
    from scipy.spatial.transform import Rotation
    Q = Rotation.random(random_state=3).as_matrix()
    QF = np.einsum("ik,kj...->ij...", Q, F)
    np.testing.assert_allclose(O.stress(QF, c, d, prm), np.einsum("ik,kj...->ij...", Q, O.stress(F, c, d, prm)),
                               rtol=1e-9, atol=1e-9 * np.abs(O.stress(F, c, d, prm)).max())
    np.testing.assert_allclose(O.psi_e(QF, c, d, prm), O.psi_e(F, c, d, prm), rtol=1e-10)


@pytest.mark.parametrize("law", LAWS)
def test_elastic_chemical_potential_is_energy_derivative(law):
    prm = params(law, omega=0.3)
    F, c, d = rand_state()
    eps = 1e-7
    fd = (O.psi_e(F, c + eps, d, prm) - O.psi_e(F, c - eps, d, prm)) / (2 * eps) / prm.cmax
    np.testing.assert_allclose(O.mu_elastic(F, c, d, prm), fd, rtol=1e-5, atol=1e-8 * np.abs(fd).max())


def test_neohooke_uniaxial_closed_form():
    """NH, F = diag(l, 1, 1): P_xx = (1-d)^2 a [G (a l - 1/(a l)) + lam ln(a^3 l)/(a l)]."""
    prm = params(O.LAW_NEOHOOKE)
    l = RNG.uniform(0.9, 1.1, SHAPE)
    c = RNG.uniform(0.05, 0.6, SHAPE)
    d = RNG.uniform(0.0, 0.5, SHAPE)
    F = np.zeros((3, 3) + SHAPE)
    F[0, 0], F[1, 1], F[2, 2] = l, 1.0, 1.0
    a = (1 + prm.Omega * (c - prm.c0)) ** (-1 / 3)
    ref = (1 - d) ** 2 * a * (prm.mu * (a * l - 1 / (a * l)) + prm.lam * np.log(a ** 3 * l) / (a * l))
    np.testing.assert_allclose(O.stress(F, c, d, prm)[0, 0], ref, rtol=1e-12)


def test_principal_stress_driving_force():
    prm = params(O.LAW_NEOHOOKE)
    from scipy.spatial.transform import Rotation
    Q = Rotation.random(random_state=5).as_matrix()
    s = np.array([150e6, 50e6, -20e6])
    sig = Q @ np.diag(s) @ Q.T
    S = np.broadcast_to(sig.reshape(3, 3, 1, 1, 1), (3, 3) + SHAPE)
    w = O.principal_stresses(S)
    np.testing.assert_allclose(np.sort(w, axis=0)[:, 0, 0, 0], np.sort(s), rtol=1e-12)
    # D_f with sigma_max = 80 MPa: (150/80)^2 + (50/80)^2 - 1
    smax = 80e6
    ref = (150 / 80) ** 2 + (50 / 80) ** 2 - 1.0
    t = np.maximum(w, 0) / smax
    assert np.allclose(np.maximum((t * t).sum(0) - 1, 0), ref)
    # the Cauchy stress of a uniaxial stretch without swelling is diag(P_xx / 1, P_yy/l, ...)
    l = 1.03
    F = np.zeros((3, 3) + SHAPE)
    F[0, 0], F[1, 1], F[2, 2] = l, 1.0, 1.0
    c = np.full(SHAPE, 0.01)
    sigma = O.cauchy_undegraded(F, c, prm)
    P = O.stress(F, c, 0 * c, prm)
    np.testing.assert_allclose(sigma[0, 0], P[0, 0] * l / l, rtol=1e-12)
    np.testing.assert_allclose(sigma[1, 1], P[1, 1] / l, rtol=1e-12)
    Df = O.driving_force(F, c, prm)
    sx = np.maximum(sigma[0, 0], 0) / prm.sigma_max
    sy = np.maximum(sigma[1, 1], 0) / prm.sigma_max
    sz = np.maximum(sigma[2, 2], 0) / prm.sigma_max
    np.testing.assert_allclose(Df, np.maximum(sx ** 2 + sy ** 2 + sz ** 2 - 1, 0), rtol=1e-12, atol=1e-14)


def test_per_voxel_strength_driving_force():
    """Per-voxel strength sigma_max(x) = sigma_max exp(log_smax) (Sec. 5.1 draws it per
    voxel): under a homogeneous uniaxial stretch the Cauchy stress is diagonal and the
    same everywhere, so D_f at each voxel is the closed form of Eq. SigDrivingForce with
    that voxel's own threshold."""
    phases = [O.Phase(law=O.LAW_SVK, E=15e9, nu=0.3, Omega=0.0, c0=0.01, sigma_max=100e6)]
    pid = np.zeros(SHAPE, dtype=int)
    log_smax = RNG.uniform(-1.5, 0.5, SHAPE)
    prm = O.make_params(phases, pid, (1e-7,) * 3, gc=1.0, lc=2e-7, log_smax=log_smax)
    np.testing.assert_allclose(prm.sigma_max, 100e6 * np.exp(log_smax), rtol=1e-15)
    l = 1.004
    F = np.zeros((3, 3) + SHAPE)
    F[0, 0], F[1, 1], F[2, 2] = l, 1.0, 1.0
    c = np.full(SHAPE, 0.01)
    # SVK: E = (l^2 - 1)/2 e1 e1, S = lam tr E I + 2 G E, sigma = F S F^T / J
    lam, G = O.lame(15e9, 0.3)
    e = 0.5 * (l * l - 1.0)
    sx = (lam * e + 2.0 * G * e) * l * l / l
    sy = lam * e / l
    thr = 100e6 * np.exp(log_smax)
    ref = np.maximum((sx / thr) ** 2 + 2.0 * (sy / thr) ** 2 - 1.0, 0.0)
    assert (ref > 0).any() and (ref == 0).any()  # both sides of the threshold
    np.testing.assert_allclose(O.driving_force(F, c, prm), ref, rtol=1e-12, atol=1e-15)
    H = O.history_update(np.zeros(SHAPE), F, c, prm)
    np.testing.assert_allclose(H, ref / (2.0 * 2e-7), rtol=1e-12)
