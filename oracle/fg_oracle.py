"""Plain CPU FP64 oracle of the FFT chemo-mechanical fracture method (arXiv 2411.16583).

TEST INFRASTRUCTURE ONLY.  This module is the independent reference that the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the
product (the ``paper_2411_16583_gb300`` package and its C-ABI library) never does,
and this module imports nothing from the product.

Everything is numpy float64, vectorised over voxels, written to be read against
the paper:

* fields are arrays ``(..., nz, ny, nx)``; a second-order tensor field is
  ``(3, 3, nz, ny, nx)`` with ``T[i, j]`` the (i, j) component;
* the DFT is numpy's: forward unnormalised with ``exp(-i q.x)``, inverse scaled by
  1/V, real-to-half-complex along x (Sec. 3.2, "Discrete Fourier Transform");
* no blocking, fusion or reordering beyond the paper's algorithms.

Readings of points the paper leaves open:

* swelling  F_c = J_c^{1/3} I with J_c = 1 + Omega (c - c0)  (Eq. Fc, shifted so the
  material is stress free at its reference concentration c0);
* the stress is the exact derivative P = d psi_e / dF of the degraded energy
  (Eq. Pderivada), i.e. P = (1-d)^2 a P0(a F) with a = J_c^{-1/3};
* mechanics uses the rotated finite-difference frequencies (Sec. 3.2, mechanical
  equilibrium), phase field and chemistry the forward/backward ones;
* the history is H = max(H_t, g_c/(2 l_c) D_f) with D_f from the undegraded Cauchy
  stress (Eqs. Hist, SigDrivingForce);
* the chemical Newton Jacobian keeps only the ideal-solution part of mu (Eq.
  Chemderfc) and is solved in the symmetric variable y = m dc, m = 1/(c(1-c)); an
  option adds the elastic part d(mu_e/RT)/dc (same root);
* toughness and strength may vary per voxel, g_c(x) = g_c exp(log_gc) and
  sigma_max(x) = sigma_max exp(log_smax) (Sec. 5.1 draws the strength per voxel).

Parity status: every function below is pinned by ``tests/test_oracle_*.py``.  The
composition of a whole coupled step (Alg. 4) is an iteration; it is pinned by the
equations its result must solve (the Fick residual with F and d frozen at the step's
start, mechanical equilibrium, the history field, the phase-field system, each through
the separately pinned functions), by a homogeneous case in closed form and by invariants
(mass balance, monotone history).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LAW_SVK = 0
LAW_NEOHOOKE = 1

# --------------------------------------------------------------------------------------
# Discrete Fourier transform and frequencies  (Sec. 3.2, "FFT resolution algorithms")
# --------------------------------------------------------------------------------------


def rfft3(a):
    """Forward DFT over the last three axes (z, y, x), unnormalised, half spectrum in x
    (Sec. 3.2, discrete Fourier transform; numpy's FFT as the library primitive)."""
    return np.fft.rfftn(a, axes=(-3, -2, -1))


def irfft3(A, shape):
    """Inverse of :func:`rfft3` (scaled by 1/V; Sec. 3.2); ``shape`` = (nz, ny, nx)."""
    return np.fft.irfftn(A, s=shape, axes=(-3, -2, -1))


def _half_angle(n, half):
    """theta_k = pi k / n for the DFT indices of one axis, with cos(theta) snapped to an
    exact 0 at the Nyquist index (2k = n), where the exact value is 0."""
    if half:
        k = np.arange(n // 2 + 1)
    else:
        k = np.rint(np.fft.fftfreq(n) * n).astype(np.int64)
    th = np.pi * k / n
    s = np.sin(th)
    c = np.cos(th)
    nyq = (2 * np.abs(k) == n)
    c[nyq] = 0.0
    s[nyq] = np.sign(k[nyq]).astype(float)
    return k, th, s, c


def _axes(shape):
    nz, ny, nx = shape
    kx = _half_angle(nx, True)
    ky = _half_angle(ny, False)
    kz = _half_angle(nz, False)
    return kz, ky, kx


def rotated_frequencies(shape, h):
    """Rotated-scheme symbol n (3, nz, ny, nx//2+1) (Sec. 3.2, mechanical equilibrium,
    rotated differentiation scheme).

    The scheme differentiates on the 2x2x2 cell of neighbouring voxels: d/dx_j is the
    mean of the four forward differences along j on that cell.  Its DFT symbol is
    i n_j exp(i sum_m q_m / 2) with n_j = (2/h_j) sin(q_j/2) prod_{m != j} cos(q_m/2).
    """
    (_, _, sz, cz), (_, _, sy, cy), (_, _, sx, cx) = _axes(shape)
    hx, hy, hz = h
    nz, ny, nx = shape
    X = (slice(None),)
    sx_, cx_ = sx[None, None, :], cx[None, None, :]
    sy_, cy_ = sy[None, :, None], cy[None, :, None]
    sz_, cz_ = sz[:, None, None], cz[:, None, None]
    if nz == 1:  # plane strain: no variation along z, q_z = 0
        sz_, cz_ = np.zeros_like(sz_), np.ones_like(cz_)
    n1 = (2.0 / hx) * sx_ * cy_ * cz_
    n2 = (2.0 / hy) * sy_ * cx_ * cz_
    n3 = (2.0 / hz) * sz_ * cx_ * cy_
    return np.stack(np.broadcast_arrays(n1, n2, n3))


def fd_frequencies(shape, h):
    """Forward finite-difference symbol xi_j = (exp(i q_j) - 1)/h_j  (3, nz, ny, nx//2+1),
    used for chemistry (Sec. 3.2, chemical problem) and the phase field Laplacian."""
    nz, ny, nx = shape
    hx, hy, hz = h
    qx = 2.0 * np.pi * np.arange(nx // 2 + 1) / nx
    qy = 2.0 * np.pi * np.rint(np.fft.fftfreq(ny) * ny) / ny
    qz = 2.0 * np.pi * np.rint(np.fft.fftfreq(nz) * nz) / nz
    x1 = ((np.exp(1j * qx) - 1.0) / hx)[None, None, :]
    x2 = ((np.exp(1j * qy) - 1.0) / hy)[None, :, None]
    x3 = ((np.exp(1j * qz) - 1.0) / hz)[:, None, None]
    return np.stack(np.broadcast_arrays(x1, x2, x3))


def fd_laplacian_symbol(shape, h):
    """|xi|^2 = sum_j 4 sin^2(q_j/2)/h_j^2 : symbol of minus the 7-point Laplacian, the xi.xi
    of Eqs. PFFA and PFFprecond under the forward-difference scheme."""
    xi = fd_frequencies(shape, h)
    return np.sum(np.abs(xi) ** 2, axis=0)


def project_G(A, n):
    """Compatibility projection in frequency space (Eq. mapping G, integral G):
    A'_ij = n_j sum_m n_m A_im / |n|^2, and 0 where |n| = 0 (the mean and the null modes
    of the rotated scheme)."""
    n2 = np.sum(n * n, axis=0)
    zero = n2 == 0.0
    inv = np.where(zero, 0.0, 1.0 / np.where(zero, 1.0, n2))
    An = np.einsum("im...,m...->i...", A, n)
    return np.einsum("i...,j...->ij...", An * inv, n)


def apply_G(T, h):
    """Real-space G * T for a real tensor field T (3,3,nz,ny,nx): F^-1[G : F[T]]
    (Eqs. mapping G, mechanicalsolve)."""
    shape = T.shape[-3:]
    n = rotated_frequencies(shape, h)
    return irfft3(project_G(rfft3(T), n), shape)


def apply_G_mixed(T, prm):
    """Projection of mixed macroscopic control: G * T plus, on the stress-controlled
    components M, the mean of T (the zero-frequency mode kept instead of removed).  It is
    the orthogonal projection onto compatible zero-mean fields plus uniform fields on M, so
    the Newton operator stays symmetric; the mean of F on M is then an unknown, with the
    mean stress on M prescribed (mixed strain/stress control of the macroscopic problem)."""
    G = apply_G(T, prm.h)
    if prm.stress_mask is None:
        return G
    mean = T.mean(axis=(2, 3, 4))
    return G + (np.where(prm.stress_mask, mean, 0.0))[:, :, None, None, None]


def stress_target(prm, shape):
    """M P-bar*: the prescribed mean stress on the controlled components, as a field
    (Sec. 3.1, macroscopic stress conditions)."""
    if prm.stress_mask is None:
        return 0.0
    return np.broadcast_to(np.where(prm.stress_mask, prm.Pbar, 0.0)[:, :, None, None, None],
                           (3, 3) + tuple(shape))


# --------------------------------------------------------------------------------------
# Tensor helpers (voxel-wise)
# --------------------------------------------------------------------------------------


def _I(like):
    eye = np.zeros((3, 3) + like.shape[2:])
    for i in range(3):
        eye[i, i] = 1.0
    return eye


def tmul(A, B):
    return np.einsum("ik...,kj...->ij...", A, B)


def tT(A):
    return np.swapaxes(A, 0, 1)


def ddot(A, B):
    return np.einsum("ij...,ij...->...", A, B)


def tdet(A):
    return (A[0, 0] * (A[1, 1] * A[2, 2] - A[1, 2] * A[2, 1])
            - A[0, 1] * (A[1, 0] * A[2, 2] - A[1, 2] * A[2, 0])
            + A[0, 2] * (A[1, 0] * A[2, 1] - A[1, 1] * A[2, 0]))


def tinv(A):
    """Inverse through numpy's LU (library routine), moving the 3x3 axes last and back."""
    M = np.moveaxis(np.moveaxis(A, 0, -1), 0, -1)  # (..., 3(i), 3(j))
    return np.moveaxis(np.moveaxis(np.linalg.inv(M), -1, 0), -1, 0)


# --------------------------------------------------------------------------------------
# Material parameters per voxel  (Sec. 2; buffer phase of Sec. 4.3 / 5.1)
# --------------------------------------------------------------------------------------


@dataclass
class Phase:
    law: int = LAW_NEOHOOKE
    E: float = 10e9
    nu: float = 0.3
    Omega: float = 0.0
    c0: float = 0.01
    D: float = 1e-14
    sigma_max: float = 100e6


@dataclass
class Params:
    """Per-voxel material arrays (nz, ny, nx) plus the global constants (Sec. 2 material
    parameters; the tables of Secs. 4.3 and 5.1)."""
    law: int
    lam: np.ndarray
    mu: np.ndarray
    Omega: np.ndarray
    c0: np.ndarray
    D: np.ndarray
    sigma_max: np.ndarray
    gc: float
    lc: float
    RT: float
    cmax: float
    h: tuple
    shape: tuple
    extra: dict = field(default_factory=dict)
    gcr: np.ndarray | None = None  # per-voxel g_c(x) / g_c (None: uniform g_c)
    stress_mask: np.ndarray | None = None  # (3, 3) bool: components of P-bar prescribed
    Pbar: np.ndarray | None = None         # (3, 3) prescribed mean stress on the mask


def gc_ratio(prm):
    """g_c(x) / g_c per voxel (ones for a uniform toughness; the paper's g_c of Eq. PFF is
    uniform)."""
    return np.ones(prm.shape) if prm.gcr is None else prm.gcr


def lame(E, nu):
    """Lame constants of Young's modulus and Poisson's ratio (Sec. 2.1)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def make_params(phases, phase_id, h, gc, lc, RT=8.314462618 * 298.15, cmax=3.0e4,
                log_E=None, log_D=None, log_gc=None, log_smax=None):
    """Gather per-phase constants onto the voxel grid (optionally times exp(log-field):
    stiffness E, diffusivity D, toughness g_c(x) = g_c exp(log_gc) and strength
    sigma_max(x) = sigma_max exp(log_smax), the per-voxel threshold of Sec. 5.1)."""
    phase_id = np.asarray(phase_id)
    laws = {p.law for p in phases}
    if len(laws) != 1:
        raise ValueError("one constitutive law for all phases")
    tab = lambda attr: np.array([getattr(p, attr) for p in phases], dtype=float)[phase_id]
    E = tab("E")
    if log_E is not None:
        E = E * np.exp(log_E)
    D = tab("D")
    if log_D is not None:
        D = D * np.exp(log_D)
    lam, mu = lame(E, tab("nu"))
    smax = tab("sigma_max")
    if log_smax is not None:
        smax = smax * np.exp(log_smax)
    return Params(law=phases[0].law, lam=lam, mu=mu, Omega=tab("Omega"), c0=tab("c0"), D=D,
                  sigma_max=smax, gc=float(gc), lc=float(lc), RT=float(RT),
                  cmax=float(cmax), h=tuple(float(x) for x in h), shape=phase_id.shape,
                  gcr=None if log_gc is None else np.exp(np.asarray(log_gc, dtype=float)))


# --------------------------------------------------------------------------------------
# Constitutive law  (Sec. 2.1, Eqs. F=Fe+Fc, Fc, Ee, psie0, psiedamaged, Pderivada)
# --------------------------------------------------------------------------------------


def swelling_J(c, prm):
    """J_c = det F_c = 1 + Omega (c - c0)  (Eq. Fc, shifted to the reference c0)."""
    return 1.0 + prm.Omega * (c - prm.c0)


def swelling_a(c, prm):
    """a = J_c^{-1/3}, so that F_e = F F_c^{-1} = a F  (Eq. F=Fe+Fc)."""
    return swelling_J(c, prm) ** (-1.0 / 3.0)


def psi0(Fe, prm):
    """Pristine elastic energy density of F_e (Eqs. Ee, psie0 for Saint-Venant-Kirchhoff;
    the compressible Neo-Hookean form for that law)."""
    if prm.law == LAW_SVK:  # Eq. psie0 with E_e = (F_e^T F_e - I)/2  (Eq. Ee)
        E = 0.5 * (tmul(tT(Fe), Fe) - _I(Fe))
        trE = E[0, 0] + E[1, 1] + E[2, 2]
        return 0.5 * prm.lam * trE ** 2 + prm.mu * ddot(E, E)
    J = tdet(Fe)  # compressible Neo-Hookean
    lnJ = np.log(J)
    return 0.5 * prm.mu * (ddot(Fe, Fe) - 3.0) - prm.mu * lnJ + 0.5 * prm.lam * lnJ ** 2


def P0(Fe, prm):
    """d psi0 / d F_e, the pristine stress of Eq. pristine."""
    if prm.law == LAW_SVK:  # Eq. pristine: F_e S,  S = lam tr(E) I + 2 G E
        E = 0.5 * (tmul(tT(Fe), Fe) - _I(Fe))
        trE = E[0, 0] + E[1, 1] + E[2, 2]
        S = prm.lam * trE * _I(Fe) + 2.0 * prm.mu * E
        return tmul(Fe, S)
    Finv_T = tT(tinv(Fe))
    lnJ = np.log(tdet(Fe))
    return prm.mu * (Fe - Finv_T) + prm.lam * lnJ * Finv_T


def dP0(Fe, dFe, prm):
    """Directional derivative d P0(F_e)[dF_e] of Eq. pristine (the tangent of Eq.
    mechanicalsolve)."""
    if prm.law == LAW_SVK:
        E = 0.5 * (tmul(tT(Fe), Fe) - _I(Fe))
        trE = E[0, 0] + E[1, 1] + E[2, 2]
        S = prm.lam * trE * _I(Fe) + 2.0 * prm.mu * E
        dE = 0.5 * (tmul(tT(Fe), dFe) + tmul(tT(dFe), Fe))
        trdE = dE[0, 0] + dE[1, 1] + dE[2, 2]
        dS = prm.lam * trdE * _I(Fe) + 2.0 * prm.mu * dE
        return tmul(dFe, S) + tmul(Fe, dS)
    Bt = tT(tinv(Fe))  # F_e^{-T}
    lnJ = np.log(tdet(Fe))
    dlnJ = ddot(Bt, dFe)
    dBt = -tmul(tmul(Bt, tT(dFe)), Bt)
    return prm.mu * (dFe - dBt) + prm.lam * (dlnJ * Bt + lnJ * dBt)


def psi_e(F, c, d, prm):
    """Degraded elastic energy (1-d)^2 psi0(a F)  (Eq. psiedamaged)."""
    a = swelling_a(c, prm)
    return (1.0 - d) ** 2 * psi0(a * F, prm)


def stress(F, c, d, prm):
    """First Piola stress P = d psi_e / dF = (1-d)^2 a P0(a F)  (Eqs. Pderivada, PFcd)."""
    a = swelling_a(c, prm)
    return (1.0 - d) ** 2 * a * P0(a * F, prm)


def tangent_apply(F, c, d, prm, dF):
    """K : dF with K = dP/dF = (1-d)^2 a^2 dP0/dF_e (a F)  (Eqs. Pderivada, mechanicalsolve)."""
    a = swelling_a(c, prm)
    return (1.0 - d) ** 2 * a * dP0(a * F, a * dF, prm)


def mu_elastic(F, c, d, prm):
    """Elastic chemical potential per mole, d psi_e/dc at fixed F divided by c_max
    (Eq. mue re-derived from Eq. psiedamaged):
    -(1-d)^2 Omega / (3 J_c) P0(F_e) : F_e / c_max."""
    a = swelling_a(c, prm)
    Fe = a * F
    Jc = swelling_J(c, prm)
    return -(1.0 - d) ** 2 * prm.Omega / (3.0 * Jc) * ddot(P0(Fe, prm), Fe) / prm.cmax


# --------------------------------------------------------------------------------------
# Damage driving force  (Eqs. Hist, SigDrivingForce)
# --------------------------------------------------------------------------------------


def cauchy_undegraded(F, c, prm):
    """sigma = J^{-1} P~ F^T with the undegraded stress P~ = a P0(a F), the stress whose
    principal values enter Eq. SigDrivingForce."""
    a = swelling_a(c, prm)
    Pu = a * P0(a * F, prm)
    s = tmul(Pu, tT(F)) / tdet(F)
    return 0.5 * (s + tT(s))


def principal_stresses(sig):
    """Eigenvalues of the symmetric 3x3 stress at every voxel (numpy eigvalsh), the
    principal stresses of Eq. SigDrivingForce."""
    M = np.moveaxis(np.moveaxis(sig, 0, -1), 0, -1)
    w = np.linalg.eigvalsh(M)
    return np.moveaxis(w, -1, 0)


def driving_force(F, c, prm):
    """D_f = < sum_i (<sigma_i>/sigma_max)^2 - 1 >, <.> the positive part
    (Eq. SigDrivingForce)."""
    s = principal_stresses(cauchy_undegraded(F, c, prm))
    t = np.maximum(s, 0.0) / prm.sigma_max
    return np.maximum(np.sum(t * t, axis=0) - 1.0, 0.0)


def history_update(H_t, F, c, prm):
    """H = max(H_t, g_c(x)/(2 l_c) D_f)  (Eq. Hist)."""
    return np.maximum(H_t, prm.gc * gc_ratio(prm) / (2.0 * prm.lc) * driving_force(F, c, prm))


# --------------------------------------------------------------------------------------
# Krylov solvers  (Alg. 1 / Alg. 2 / Alg. 3 name conjugate gradients)
# --------------------------------------------------------------------------------------


def dot(a, b):
    return float(np.vdot(a.ravel(), b.ravel()).real)


def cg(apply, b, tol, maxit, x0=None, stats=None, indefinite=True, info=None):
    """Textbook conjugate gradients (the linear solver of Algs. 1 and 3); stops when
    ||r|| <= tol ||b||.  Returns (x, iters).

    Near a prestressed equilibrium the mechanical tangent of a particle in a soft buffer
    is not always positive definite.  With indefinite=True a direction of negative
    curvature <p, Ap> < 0 is taken like any other (the Galerkin iterate of the symmetric
    system exists while <p, Ap> != 0); with indefinite=False CG stops at the first one and
    keeps its iterate (truncated CG).  <p, Ap> = 0 or a non-finite value always stops.
    The iterate is saved each time |r|^2 falls to a quarter of the last saved value (the
    first time: of |b - A x0|^2); a solve that stops early (truncation or maxit) after
    saving one returns the saved iterate when its own residual is larger.  With an `info`
    dict a stop at non-positive curvature returns at once and leaves in info the Rayleigh
    quotients rq = <p, Ap>/|p|^2 of that direction and rq0 = <b, Ab>/|b|^2."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply(x) if x0 is not None else b.copy()
    bn = math.sqrt(dot(b, b))
    if bn == 0.0:
        return np.zeros_like(b), 0
    p = r.copy()
    rr = dot(r, r)
    rr_best, x_best = rr, None
    it = 0
    rq0 = None
    while math.sqrt(rr) > tol * bn and it < maxit:
        q = apply(p)
        pq = dot(p, q)
        if rq0 is None:
            rq0 = pq / dot(p, p)
        if info is not None and not pq > 0.0 and not (indefinite and pq < 0.0):
            info["rq"] = pq / dot(p, p)
            info["rq0"] = rq0
            return x, it
        if indefinite and pq < 0.0:
            if stats is not None:
                stats["cg_negcurv"] = stats.get("cg_negcurv", 0) + 1
        elif not pq > 0.0:
            if it == 0:
                raise FloatingPointError("operator not positive along the residual")
            if stats is not None:
                stats["cg_truncated"] = stats.get("cg_truncated", 0) + 1
            break
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = dot(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        if rr <= 0.25 * rr_best:
            rr_best, x_best = rr, x.copy()
    if x_best is not None and math.sqrt(rr) > tol * bn and rr > rr_best:
        x = x_best
    return x, it


def shifted_cg(apply, b, tol, maxit, stats=None):
    """CG on the Newton system, shifted where it is not positive definite: a solve that
    meets a direction p with <p, (A + sigma) p> <= 0 sets sigma to 2 (sigma + |rq|), rq
    its Rayleigh quotient (|rq| at least 1e-6 |<b, Ab>|/|b|^2), and starts again from
    zero, until a solve meets none (at most 13 solves).  A Rayleigh quotient only bounds
    the lowest eigenvalue from above, so the shift grows geometrically instead of
    stopping just above it, where the system would be nearly singular.
    Returns (x, iterations, sigma)."""
    sigma, its = 0.0, 0
    for _ in range(13):
        info = {}
        x, it = cg(lambda v: apply(v) + sigma * v, b, tol, maxit, stats=stats,
                   indefinite=False, info=info)
        its += it
        if "rq" not in info:
            return x, its, sigma
        sigma = 2.0 * (sigma + max(abs(info["rq"]), 1e-6 * abs(info["rq0"])))
        if stats is not None:
            stats["newton_shifted"] = stats.get("newton_shifted", 0) + 1
    raise FloatingPointError("shifted system still not positive")


def minres(apply, b, tol, maxit, stats=None):
    """MINRES (Paige and Saunders 1975) for a symmetric, possibly indefinite operator, from
    x = 0 until |b - A x| <= tol |b|.  Lanczos: A v_k = b_k v_{k-1} + a_k v_k + b_{k+1} v_{k+1}
    (b_1 = 0 in column 1).  Column k of the tridiagonal matrix, (b_k, a_k, b_{k+1}) in rows
    k-1, k, k+1, is rotated by the Givens rotations G_{k-2}, G_{k-1} into (e_k, d_k, gbar_k)
    plus b_{k+1}, which G_k = (c, s) = (gbar_k, b_{k+1}) / gamma_k removes; the rotated
    right-hand side gives phi_k = c phibar_{k-1}, phibar_k = -s phibar_{k-1}, |phibar_k| the
    residual norm, and x_k = x_{k-1} + phi_k w_k with w_k = (v_k - d_k w_{k-1} - e_k w_{k-2})
    / gamma_k.  Returns (x, iterations)."""
    x = np.zeros_like(b)
    beta1 = math.sqrt(dot(b, b))
    if beta1 == 0.0:
        return x, 0
    v_prev = np.zeros_like(b)
    v = b / beta1
    beta = 0.0  # b_k, the coupling of v_k to v_{k-1}
    w1 = np.zeros_like(b)  # w_{k-1}
    w2 = np.zeros_like(b)  # w_{k-2}
    c1, s1, c2, s2 = 1.0, 0.0, 1.0, 0.0  # G_{k-1}, G_{k-2}
    phibar = beta1
    it = 0
    while abs(phibar) > tol * beta1 and it < maxit:
        Av = apply(v)
        alpha = dot(v, Av)
        u = Av - alpha * v - beta * v_prev
        beta_next = math.sqrt(dot(u, u))
        e = s2 * beta
        t = c2 * beta
        d = c1 * t + s1 * alpha
        gbar = -s1 * t + c1 * alpha
        gamma = math.hypot(gbar, beta_next)
        c, s = (gbar / gamma, beta_next / gamma) if gamma > 0.0 else (1.0, 0.0)
        phi = c * phibar
        phibar = -s * phibar
        w = (v - d * w1 - e * w2) / gamma
        x = x + phi * w
        w2, w1 = w1, w
        c2, s2, c1, s1 = c1, s1, c, s
        it += 1
        if beta_next == 0.0:
            break
        v_prev, v, beta = v, u / beta_next, beta_next
    if stats is not None:
        stats["minres"] = stats.get("minres", 0) + it
    return x, it


def pcg(apply, precond, b, tol, maxit, x0):
    """Preconditioned conjugate gradients from x0 (Alg. 2); stops when ||r|| <= tol ||b||."""
    bn = math.sqrt(dot(b, b))
    if bn == 0.0:
        return np.zeros_like(b), 0
    x = x0.copy()
    r = b - apply(x)
    z = precond(r)
    p = z.copy()
    rz = dot(r, z)
    it = 0
    while math.sqrt(dot(r, r)) > tol * bn and it < maxit:
        q = apply(p)
        alpha = rz / dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        z = precond(r)
        rz_new = dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it


# --------------------------------------------------------------------------------------
# Mechanics  (Eqs. mechanicalsolve, mechresiduum; Alg. 1)
# --------------------------------------------------------------------------------------


def mech_apply(F, c, d, prm, dF):
    """One matrix-free operator application  F^-1[ G : F[K : dF] ] (Eq. mechanicalsolve;
    G of mixed control when stress components are prescribed)."""
    return apply_G_mixed(tangent_apply(F, c, d, prm, dF), prm)


def mech_residual(F, c, d, prm, Fbar):
    """Returns (G*P(F), err_res) with err_res = ||G*P(F)|| / ||G*P(Fbar)|| (Eq. mechresiduum).

    When the comparison stress has no incompatible part (a homogeneous medium) the
    denominator falls back to ||P(Fbar)||, then to 1."""
    GP = apply_G_mixed(stress(F, c, d, prm), prm) - stress_target(prm, F.shape[2:])
    Fb = np.broadcast_to(np.asarray(Fbar, dtype=float).reshape(3, 3, 1, 1, 1), F.shape)
    Pb = stress(np.array(Fb), c, d, prm)
    GPb = apply_G_mixed(Pb, prm) - stress_target(prm, F.shape[2:])
    den = math.sqrt(dot(GPb, GPb))
    nPb = math.sqrt(dot(Pb, Pb))
    if den <= 1e-12 * nPb:
        den = nPb
    if den == 0.0:
        den = 1.0
    return GP, math.sqrt(dot(GP, GP)) / den


def mech_newton(F, c, d, prm, Fbar, tol_newton, tol_cg, max_newton, max_cg, stats=None,
                indefinite=2):
    """Alg. 1 from the given F (the caller sets F^0 = F_t + dFbar).

    indefinite selects what a CG direction of negative curvature does: 2 = the shifted
    re-solve of shifted_cg, with the shift of the previous Newton iteration divided by 4 as
    the starting shift; 1 = CG takes it; 0 = truncated CG.

    Each Newton correction dF is damped, lambda = 1, 1/2, ... (at most 10 halvings),
    until F + lambda dF stays in the domain (det F > 0, J_c > 0) and lowers err_res.  When a
    CG correction fails that (the tangent of the current state has negative eigenvalues
    along which a shifted or truncated direction cannot lower the residual), the iteration
    is redone with MINRES on the unshifted Newton system, and MINRES serves the rest of
    the solve."""
    n_newton = 0
    sigma = 0.0
    use_minres = False
    GP, err = mech_residual(F, c, d, prm, Fbar)
    while True:
        if stats is not None:
            stats.setdefault("err_mech", []).append(err)
        if err <= tol_newton:
            return F, err
        if n_newton >= max_newton:
            raise RuntimeError("mechanical Newton did not converge")
        if use_minres:
            dF, it = minres(lambda x: mech_apply(F, c, d, prm, x), -GP, tol_cg, max_cg, stats)
        elif indefinite == 2:
            s0 = sigma / 4.0
            dF, it, sigma = shifted_cg(lambda x: mech_apply(F, c, d, prm, x) + s0 * x, -GP,
                                       tol_cg, max_cg, stats)
            sigma += s0
        else:
            dF, it = cg(lambda x: mech_apply(F, c, d, prm, x), -GP, tol_cg, max_cg,
                        stats=stats, indefinite=bool(indefinite))
        n_newton += 1
        if stats is not None:
            stats["newton_mech"] = stats.get("newton_mech", 0) + 1
            stats["cg_mech"] = stats.get("cg_mech", 0) + it
        lam = 1.0
        for _ in range(11):
            Fn = F + lam * dF
            ok = bool(np.all(tdet(Fn) > 0.0)) and bool(np.all(swelling_J(c, prm) > 0.0))
            if ok:
                with np.errstate(all="ignore"):
                    GPn, errn = mech_residual(Fn, c, d, prm, Fbar)
                if errn < err:
                    break
            if stats is not None:
                stats["newton_damped"] = stats.get("newton_damped", 0) + 1
            lam *= 0.5
        else:
            if use_minres:
                raise RuntimeError("mechanical Newton: no decrease of err_res along the correction")
            use_minres = True
            if stats is not None:
                stats["newton_minres"] = stats.get("newton_minres", 0) + 1
            continue
        F, GP, err = Fn, GPn, errn


def mech_adjoint(F, c, d, prm, W, tol_cg, max_cg):
    """Gradient with respect to the per-voxel log stiffness of a loss L(F) with dL/dF = W,
    at an equilibrium G*P(F) = 0 (Eq. mechanicalsolve): with lambda solving the transposed
    tangent system G K G lambda = G W (K is symmetric) and dP/dlogE = P at fixed F,
    dL/dlogE(v) = -lambda(v) : P(v)."""
    lam, _ = cg(lambda x: mech_apply(F, c, d, prm, x), apply_G(W, prm.h), tol_cg, max_cg)
    return -np.sum(lam * stress(F, c, d, prm), axis=(0, 1))


# --------------------------------------------------------------------------------------
# Phase field  (Eqs. PFFrearranged, PFFA, PFFb, PFFprecond; Alg. 2)
# --------------------------------------------------------------------------------------


def pff_apply(dd, H, prm):
    """A(d) = [g_c/l_c + 2H] d + F^-1{ g_c l_c |xi|^2 d^ }  (Eq. PFFA)."""
    lap = fd_laplacian_symbol(prm.shape, prm.h)
    return (prm.gc / prm.lc + 2.0 * H) * dd + irfft3(prm.gc * prm.lc * lap * rfft3(dd), prm.shape)


def pff_precond(r, Hbar, prm):
    """P(r) = F^-1{ r^ / (g_c/l_c + 2 Hbar + g_c l_c |xi|^2) }  (Eq. PFFprecond)."""
    lap = fd_laplacian_symbol(prm.shape, prm.h)
    return irfft3(rfft3(r) / (prm.gc / prm.lc + 2.0 * Hbar + prm.gc * prm.lc * lap), prm.shape)


def pff_solve(H, d0, prm, tol, maxit, stats=None):
    """Alg. 2.  With a per-voxel toughness g_c(x) the strong form
    g_c(x) (d/l_c - l_c lap d) = 2 (1 - d) H is divided by g_c(x)/g_c, which keeps the
    symmetric operator of Eq. PFFA with H replaced by H g_c / g_c(x)."""
    Heff = H / gc_ratio(prm)
    Hbar = float(np.mean(Heff))
    d, it = pcg(lambda x: pff_apply(x, Heff, prm), lambda r: pff_precond(r, Hbar, prm),
                2.0 * Heff, tol, maxit, d0)
    if stats is not None:
        stats["cg_pff"] = stats.get("cg_pff", 0) + it
    return d


# --------------------------------------------------------------------------------------
# Chemistry  (Eqs. ChemDTsolve, Chemresidualfc, Chemderfc, newton, Chemerror; Alg. 3)
# --------------------------------------------------------------------------------------


def mobility_phi(d):
    """Damage factor of the mobility, M = -(D/RT) phi(d)  (Eq. mobility)."""
    return 0.9 * (1.0 - d) ** 2 + 0.1 * d ** 2


def chem_conductivity(F_t, c_t, d_t, prm):
    """K_c = D phi(d_t) c_t (1 - c_t) C_t^{-1}  (3,3,...), the semi-implicit mobility of
    Eq. ChemDTsolve with RT cancelled against mu = RT mu~."""
    Cinv = tinv(tmul(tT(F_t), F_t))
    return prm.D * mobility_phi(d_t) * c_t * (1.0 - c_t) * Cinv


def chem_L(u, Kc, prm):
    """L u = grad_f^H (K_c grad_f u): minus the discrete divergence of K_c grad u, with
    forward differences for the gradient and their adjoint for the divergence (Eq.
    ChemresidualFourier_A)."""
    xi = fd_frequencies(prm.shape, prm.h)
    U = rfft3(u)
    g = irfft3(xi * U[None], prm.shape)  # (3, ...) forward-difference gradient
    flux = np.einsum("jl...,l...->j...", Kc, g)
    return irfft3(np.sum(np.conj(xi) * rfft3(flux), axis=0), prm.shape)


def chem_potential(c, F, d, prm):
    """mu~ = mu / RT = log(c/(1-c)) + mu_e / RT  (Eqs. muc, mue)."""
    return np.log(c / (1.0 - c)) + mu_elastic(F, c, d, prm) / prm.RT


def chem_residual(c, c_t, F, d_t, Kc, dt, cdot_B, prm):
    """f(c) = c - c_t + dt L mu~(c) - dt cdot_B  (Eq. Chemresidualfc)."""
    return c - c_t + dt * chem_L(chem_potential(c, F, d_t, prm), Kc, prm) - dt * cdot_B


def chem_apply(y, m, Kc, dt, prm):
    """Symmetric Newton operator in y = m dc: y/m + dt L y  (Eq. Chemderfc with
    m = mu_c'/RT = 1/(c(1-c)))."""
    return y / m + dt * chem_L(y, Kc, prm)


def chem_jacobian_elastic(c, F, d, prm):
    """d(mu_e/RT)/dc at fixed F, d: (1-d)^2 Omega^2/(3 c_max J_c^2 RT) (q + (K0[F_e]:F_e + q)/3),
    q = P0(F_e) : F_e (the derivative of Eq. mue in c)."""
    a = swelling_a(c, prm)
    Jc = swelling_J(c, prm)
    Fe = a * F
    q = ddot(P0(Fe, prm), Fe)
    kf = ddot(dP0(Fe, Fe, prm), Fe)
    return (1.0 - d) ** 2 * prm.Omega ** 2 / (3.0 * prm.cmax * Jc ** 2 * prm.RT) * (q + (kf + q) / 3.0)


def chem_solve(c_t, F, d_t, dt, cdot_B, prm, tol_chem, tol_cg, max_newton, max_cg, stats=None,
               full_jacobian=False):
    """Alg. 3: Newton-CG from c^0 = c_t until ||dc|| / ||c_t|| < tol_chem.  A correction
    that would take c out of (0, 1), where mu_c = RT log(c/(1-c)) is undefined, is halved
    (at most 10 times) until the update stays inside.  full_jacobian adds the elastic part
    of dmu~/dc to the Jacobian, which the paper's Newton leaves out (same root)."""
    Kc = chem_conductivity(F, c_t, d_t, prm)
    c = c_t.copy()
    nct = math.sqrt(dot(c_t, c_t))
    for k in range(max_newton):
        f = chem_residual(c, c_t, F, d_t, Kc, dt, cdot_B, prm)
        m = 1.0 / (c * (1.0 - c))
        if full_jacobian:  # the elastic part of dmu~/dc as well (Alg. 3 keeps mu_c' only)
            m = m + chem_jacobian_elastic(c, F, d_t, prm)
            if not np.all(m > 0.0):
                raise FloatingPointError("chemistry Jacobian not positive (dmu~/dc <= 0)")
        y, it = cg(lambda v: chem_apply(v, m, Kc, dt, prm), -f, tol_cg, max_cg)
        dc = y / m
        for _ in range(11):
            cn = c + dc
            if np.all(cn > 0.0) and np.all(cn < 1.0):
                break
            dc = 0.5 * dc
        else:
            raise FloatingPointError("concentration left (0, 1)")
        c = cn
        if stats is not None:
            stats["newton_chem"] = stats.get("newton_chem", 0) + 1
            stats["cg_chem"] = stats.get("cg_chem", 0) + it
        if math.sqrt(dot(dc, dc)) / nct < tol_chem:
            return c
    raise RuntimeError("chemical Newton did not converge")


# --------------------------------------------------------------------------------------
# Global staggered scheme  (Alg. 4)
# --------------------------------------------------------------------------------------


@dataclass
class Tolerances:
    tol_newton: float = 1e-9
    tol_cg: float = 1e-10
    tol_chem: float = 1e-9
    tol_chem_cg: float = 1e-10
    tol_pff_cg: float = 1e-10
    tol_stag: float = 1e-9
    max_newton: int = 30
    max_cg: int = 5000
    max_chem_newton: int = 50
    max_stag: int = 50
    cg_indefinite: int = 2
    chem_full_jacobian: bool = False


class CoupledState:
    """Fields (F, c, d, H) at the last converged time step and the staggered step of
    Alg. 4.  Initial state: F = I, d = 0, H = 0, c = c_init (Alg. 4 data)."""

    def __init__(self, prm, c_init, cdot_B, tol=None):
        self.prm = prm
        shp = prm.shape
        self.F = np.zeros((3, 3) + shp)
        for i in range(3):
            self.F[i, i] = 1.0
        self.c = np.array(c_init, dtype=float).reshape(shp)
        self.d = np.zeros(shp)
        self.H = np.zeros(shp)
        self.cdot_B = np.array(cdot_B, dtype=float).reshape(shp)
        self.Fbar = np.eye(3)
        self.tol = tol or Tolerances()

    def step(self, dt, Fbar_new):
        prm, tol = self.prm, self.tol
        stats = {}
        Fbar_new = np.asarray(Fbar_new, dtype=float).reshape(3, 3)
        dFbar = (Fbar_new - self.Fbar).reshape(3, 3, 1, 1, 1)
        F_t, c_t, d_t, H_t = self.F, self.c, self.d, self.H
        F = F_t + dFbar  # F_{t+dt} = Fbar_{t+dt} + F~_t
        c = chem_solve(c_t, F, d_t, dt, self.cdot_B, prm, tol.tol_chem, tol.tol_chem_cg,
                       tol.max_chem_newton, tol.max_cg, stats, tol.chem_full_jacobian)
        d = d_t.copy()
        H = H_t.copy()
        stag = 0
        # Alg. 4 evaluates err_res inside the body of its loop, so the body (mechanics,
        # history, phase field) runs at least once per step, also when the step starts in
        # equilibrium (an affine load of a homogeneous medium); the loop then ends once the
        # state (F, c, d) it left is in equilibrium
        while True:
            _, err = mech_residual(F, c, d, prm, Fbar_new)
            stats.setdefault("err_stag", []).append(err)
            if err <= tol.tol_stag and stag > 0:
                break
            if stag >= tol.max_stag:
                raise RuntimeError("staggered scheme did not converge")
            F, _ = mech_newton(F, c, d, prm, Fbar_new, tol.tol_newton, tol.tol_cg,
                               tol.max_newton, tol.max_cg, stats, tol.cg_indefinite)
            H = history_update(H_t, F, c, prm)
            d = pff_solve(H, d, prm, tol.tol_pff_cg, tol.max_cg, stats)
            stag += 1
        stats["stag"] = stag
        if prm.stress_mask is not None:  # the controlled components of F-bar were unknowns
            Fbar_new = np.where(prm.stress_mask, F.mean(axis=(2, 3, 4)), Fbar_new)
        self.F, self.c, self.d, self.H, self.Fbar = F, c, d, H, Fbar_new
        return stats


def crack_energy(d, prm, gc_field=None):
    """Fracture energy  sum_voxels g_c (d^2/(2 l_c) + l_c/2 |grad_f d|^2) h^3  (Eq. crack)."""
    xi = fd_frequencies(prm.shape, prm.h)
    g = irfft3(xi * rfft3(d)[None], prm.shape)
    gc = prm.gc * gc_ratio(prm) if gc_field is None else gc_field
    dens = gc * (d * d / (2.0 * prm.lc) + 0.5 * prm.lc * np.sum(g * g, axis=0))
    return float(np.sum(dens) * prm.h[0] * prm.h[1] * prm.h[2])
