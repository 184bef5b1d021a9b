"""Discrete adjoint of the staggered time step (Alg. 4) -- TEST INFRASTRUCTURE ONLY.

Plain numpy FP64, written from the forward equations of fg_oracle, which this module
differentiates by hand.  Nothing in the product imports it; tests, the package's
`smoke()` and the benchmark's CPU baseline do.

One converged step maps the state (c_t, F_t, d_t, H_t) to (c, F, d, H) through
  chemistry  f(c) = c - c_t + dt L_K mu~(c, F~, d_t) - dt cdot_B = 0
             (Eq. Chemresidualfc, K = K_c(F~, c_t, d_t), F~ = F_t + Fbar - Fbar_t),
  mechanics  G P(F, c, d) = 0 with F - Fbar compatible            (Eq. mechanicalsolve),
  history    H = max(H_t, psi(F, c)),  psi = g_c(x)/(2 l_c) D_f     (Eqs. Hist, SigDrivingForce),
  phase      (g_c/l_c + 2 r H) d - g_c l_c lap d - 2 r H = 0,  r = g_c/g_c(x)   (Eq. PFFA).
The reverse step takes the seeds dL/d(c, F, d, H) of the outputs and returns the seeds of
the inputs plus dL/d(log E, log g_c, log D) per voxel:
  * the (F, H, d) block by transposed block Gauss-Seidel sweeps (G K G and the
    phase-field operator are symmetric; the couplings are dP/dd and dpsi/dF on the active
    branch chi = [psi > H_t] of the max), accelerated by GMRES on the phase-field
    multiplier,
  * the chemistry by its exact Jacobian transpose I + dt M L with M = dmu~/dc, solved
    as the symmetric system (M^-1 + dt L) y = M^-1 g (the forward Newton of Alg. 3 uses
    only the ideal part of M; its root is the same).

Parity pins: tests/test_oracle_adjoint.py (central differences of the forward).
"""
import math

import numpy as np

from oracle import fg_oracle as O


# --------------------------------------------------------------------------------------
# Pointwise derivatives
# --------------------------------------------------------------------------------------


def _sym_positive_part(sig):
    """<sigma>_+ = sum_i max(s_i, 0) n_i n_i^T of symmetric 3x3 fields (numpy eigh)."""
    M = np.moveaxis(np.moveaxis(sig, 0, -1), 0, -1)
    w, Q = np.linalg.eigh(M)
    Pp = np.einsum("...ik,...k,...jk->...ij", Q, np.maximum(w, 0.0), Q)
    return np.moveaxis(np.moveaxis(Pp, -1, 0), -1, 0)


def stress_dc(F, c, d, prm):
    """dP/dc at fixed F, d: (1-d)^2 (da/dc) (P0(F_e) + K0(F_e)[F_e]), da/dc = -a Omega/(3 J_c)."""
    a = O.swelling_a(c, prm)
    Jc = O.swelling_J(c, prm)
    Fe = a * F
    da = -a * prm.Omega / (3.0 * Jc)
    return (1.0 - d) ** 2 * da * (O.P0(Fe, prm) + O.dP0(Fe, Fe, prm))


def stress_dd(F, c, d, prm):
    """dP/dd = -2 (1-d) a P0(a F)."""
    a = O.swelling_a(c, prm)
    return -2.0 * (1.0 - d) * a * O.P0(a * F, prm)


def psi_terms(F, c, prm):
    """psi = g_c(x)/(2 l_c) D_f(sigma(F, c)) and its derivatives.

    With S = dpsi/dsigma = g_c(x)/(2 l_c) [D_f > 0] (2/sigma_max^2) <sigma>_+ (the gradient
    of sum_i <s_i>^2 is the matrix function 2<sigma>_+) and sigma = sym(P~ F^T)/J,
    P~ = a P0(a F):
      dpsi/dF = (a^2 K0(F_e)[S F] + S P~)/J - (S : sigma) F^-T,
      dpsi/dc = (S F) : (dP~/dc) / J,   dP~/dc = (da/dc)(P0 + K0[F_e]),
      dpsi/dlog E = S : sigma   (sigma is proportional to E at fixed F, c).
    Returns (psi, dpsi/dF, dpsi/dc, dpsi/dlogE)."""
    a = O.swelling_a(c, prm)
    Jc = O.swelling_J(c, prm)
    Fe = a * F
    P0 = O.P0(Fe, prm)
    Pt = a * P0
    J = O.tdet(F)
    sig = O.cauchy_undegraded(F, c, prm)
    Df = O.driving_force(F, c, prm)
    scale = prm.gc * O.gc_ratio(prm) / (2.0 * prm.lc)
    psi = scale * Df
    S = (scale * (Df > 0.0) * 2.0 / prm.sigma_max ** 2) * _sym_positive_part(sig)
    SF = O.tmul(S, F)
    Z = (a * a * O.dP0(Fe, SF, prm) + O.tmul(S, Pt)) / J - O.ddot(S, sig) * O.tT(O.tinv(F))
    dPt_dc = (-a * prm.Omega / (3.0 * Jc)) * (P0 + O.dP0(Fe, Fe, prm))
    psi_c = O.ddot(SF, dPt_dc) / J
    psi_E = O.ddot(S, sig)
    return psi, Z, psi_c, psi_E


def mu_elastic_derivs(F, c, d, prm):
    """mu_e = -(1-d)^2 Omega/(3 J_c c_max) q, q = P0(F_e) : F_e, and
      dmu_e/dF = -(1-d)^2 Omega/(3 J_c c_max) a (K0[F_e] + P0),
      dmu_e/dc = (1-d)^2 Omega^2/(3 c_max J_c^2) (q + (K0[F_e] : F_e + q)/3),
      dmu_e/dd = -2/(1-d) mu_e,   dmu_e/dlog E = mu_e.
    Returns (mu_e, dmu_e/dF, dmu_e/dc)."""
    a = O.swelling_a(c, prm)
    Jc = O.swelling_J(c, prm)
    Fe = a * F
    P0 = O.P0(Fe, prm)
    KFe = O.dP0(Fe, Fe, prm)
    q = O.ddot(P0, Fe)
    g = (1.0 - d) ** 2
    pre = -g * prm.Omega / (3.0 * Jc * prm.cmax)
    mue = pre * q
    dF = pre * a * (KFe + P0)
    dc = g * prm.Omega ** 2 / (3.0 * prm.cmax * Jc ** 2) * (q + (O.ddot(KFe, Fe) + q) / 3.0)
    return mue, dF, dc


def conductivity_form_dF(F, c_t, d_t, gl, gm, prm):
    """d/dF of s = gl^T K_c(F) gm with K_c = kappa C^-1, C = F^T F, kappa = D phi c_t(1-c_t):
    ds/dF_ij = -kappa [(F w)_i u_j + (F u)_i w_j],  u = C^-1 gl, w = C^-1 gm."""
    Ci = O.tinv(O.tmul(O.tT(F), F))
    kappa = prm.D * O.mobility_phi(d_t) * c_t * (1.0 - c_t)
    u = np.einsum("ij...,j...->i...", Ci, gl)
    w = np.einsum("ij...,j...->i...", Ci, gm)
    Fu = np.einsum("ij...,j...->i...", F, u)
    Fw = np.einsum("ij...,j...->i...", F, w)
    return -kappa * (np.einsum("i...,j...->ij...", Fw, u) + np.einsum("i...,j...->ij...", Fu, w))


def fd_gradient(u, prm):
    """grad_f u (3, ...): the forward-difference gradient of the chemistry operator."""
    xi = O.fd_frequencies(prm.shape, prm.h)
    return O.irfft3(xi * O.rfft3(u)[None], prm.shape)


def fd_divergence_adj(f, prm):
    """grad_f^H f: the transpose of fd_gradient (minus the discrete divergence)."""
    xi = O.fd_frequencies(prm.shape, prm.h)
    return O.irfft3(np.sum(np.conj(xi) * O.rfft3(f), axis=0), prm.shape)


def gmres(apply, b, tol, maxit):
    """Unrestarted GMRES from x = 0 (Arnoldi with modified Gram-Schmidt, the small least
    squares problem solved by numpy) until ||b - A x|| <= tol ||b||.  Returns (x, iters)."""
    beta = math.sqrt(O.dot(b, b))
    if beta == 0.0:
        return np.zeros_like(b), 0
    Q = [b / beta]
    Hm = np.zeros((maxit + 1, maxit))
    for k in range(maxit):
        w = apply(Q[k])
        for j in range(k + 1):
            Hm[j, k] = O.dot(Q[j], w)
            w = w - Hm[j, k] * Q[j]
        Hm[k + 1, k] = math.sqrt(O.dot(w, w))
        e1 = np.zeros(k + 2)
        e1[0] = beta
        y = np.linalg.lstsq(Hm[:k + 2, :k + 1], e1, rcond=None)[0]
        res = np.linalg.norm(Hm[:k + 2, :k + 1] @ y - e1)
        if res <= tol * beta or Hm[k + 1, k] == 0.0:
            return sum(y[j] * Q[j] for j in range(k + 1)), k + 1
        Q.append(w / Hm[k + 1, k])
    raise RuntimeError("GMRES did not converge")


# --------------------------------------------------------------------------------------
# Trajectory and reverse step
# --------------------------------------------------------------------------------------


class Snapshot:
    """State after a step: c, F, d, H, the macroscopic Fbar it stores (under mixed control
    the mean of F on the stress-controlled components) and Fcmd, the Fbar the step was
    called with (equal to Fbar without mixed control)."""

    def __init__(self, c, F, d, H, Fbar, Fcmd=None):
        self.c, self.F, self.d, self.H = c.copy(), F.copy(), d.copy(), H.copy()
        self.Fbar = np.array(Fbar, dtype=float).reshape(3, 3)
        self.Fcmd = self.Fbar.copy() if Fcmd is None else np.array(Fcmd, dtype=float).reshape(3, 3)
        # a state left by a step stores mean(F) on the stress-controlled components as Fbar
        self.mean_controlled = Fcmd is not None


def forward(prm, c_init, cdot_B, dts, Fbars, tol):
    """Runs Alg. 4 from the initial state and returns the nsteps + 1 snapshots."""
    st = O.CoupledState(prm, c_init, cdot_B, tol)
    traj = [Snapshot(st.c, st.F, st.d, st.H, st.Fbar)]
    for dt, Fb in zip(dts, Fbars):
        st.step(dt, Fb)
        traj.append(Snapshot(st.c, st.F, st.d, st.H, st.Fbar, Fb))
    return traj


def crack_energy_seed(d, prm):
    """Gamma_E(d) = sum g_c(x) (d^2/(2 l_c) + l_c/2 |grad_f d|^2) h^3 (Eq. crack), its
    gradient dGamma/dd = h^3 (g_c(x) d / l_c + l_c grad_f^H (g_c(x) grad_f d)) and the
    direct part of dGamma/dlog g_c (the density itself).  Returns (value, seed_d, grad_gc)."""
    h3 = prm.h[0] * prm.h[1] * prm.h[2]
    gcx = prm.gc * O.gc_ratio(prm)
    g = fd_gradient(d, prm)
    dens = gcx * (d * d / (2.0 * prm.lc) + 0.5 * prm.lc * np.sum(g * g, axis=0)) * h3
    seed = h3 * (gcx * d / prm.lc + prm.lc * fd_divergence_adj(gcx * g, prm))
    return float(np.sum(dens)), seed, dens


def displacement_multiplier(prm):
    """m_j(k) = -i exp(-i sum_m q_m/2) n_j / |n|^2, and 0 where |n| = 0: the least-squares
    inverse of the rotated-scheme gradient of a field at the voxel corners, whose DFT
    symbol is i n_j exp(i sum_m q_m/2) (Sec. 3.2, rotated scheme; n of
    fg_oracle.rotated_frequencies).  Shape (3, nz, ny, nx//2+1)."""
    shape = prm.shape
    n = O.rotated_frequencies(shape, prm.h)
    (_, _, sz, cz), (_, _, sy, cy), (_, _, sx, cx) = O._axes(shape)
    if shape[0] == 1:  # plane strain: q_z = 0
        sz, cz = np.zeros_like(sz), np.ones_like(cz)
    e = ((cx - 1j * sx)[None, None, :] * (cy - 1j * sy)[None, :, None]
         * (cz - 1j * sz)[:, None, None])
    nn = np.sum(n * n, axis=0)
    inv = np.divide(1.0, nn, out=np.zeros_like(nn), where=nn > 0.0)
    return -1j * e[None] * n * inv[None]


def corner_nodes(prm):
    """Positions x_j = i_j h_j of the voxel corners (3, nz, ny, nx); corner i is the lower
    corner of voxel i."""
    nz, ny, nx = prm.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([x * prm.h[0], y * prm.h[1], z * prm.h[2]]).astype(float)


def corner_displacement(F, Fbar, prm):
    """Displacement at the voxel corners, u = (Fbar - I) x + u~, from the split F =
    Fbar + grad u~ (Eq. Fsplit): u~ periodic with zero mean, and its rotated-scheme
    gradient equal to F - mean(F) in least squares (exactly, for a compatible F, up to the
    scheme's null modes)."""
    m = displacement_multiplier(prm)
    Uh = np.einsum("j...,ij...->i...", m, O.rfft3(F))
    u = O.irfft3(Uh, prm.shape)
    A = np.asarray(Fbar, dtype=float).reshape(3, 3) - np.eye(3)
    return u + np.einsum("ij,j...->i...", A, corner_nodes(prm))


def corner_displacement_adjoint(r, prm):
    """Transpose of F -> u~ of corner_displacement: sum_i <u~_i, r_i> = sum_ij <F_ij, g_ij>
    for g = irfft3(conj(m_j) rfft3(r_i)) (unnormalised forward DFT, 1/V inverse)."""
    m = displacement_multiplier(prm)
    G = np.conj(m)[None] * O.rfft3(r)[:, None]
    return O.irfft3(G, prm.shape)


def displacement_mismatch(F, Fbar, u_obs, w, prm):
    """L = 1/2 sum_corners w |u - u_obs|^2 h^3 with u = corner_displacement(F, Fbar) and
    its seed dL/dF (3, 3, ...).  Returns (L, seed_F)."""
    h3 = prm.h[0] * prm.h[1] * prm.h[2]
    diff = corner_displacement(F, Fbar, prm) - u_obs
    r = w[None] * diff * h3
    return 0.5 * float(np.sum(w[None] * diff * diff)) * h3, corner_displacement_adjoint(r, prm)


def step_adjoint(prm, s_in, s_out, dt, seeds, tol, stats=None):
    """Reverse of one converged step.  seeds = dict(c, F, d, H) of dL/d(outputs); returns
    (dict(c, F, d, H) of dL/d(inputs), dict(E, gc, D) of dL/dlog-parameters)."""
    c_t, F_t, d_t, H_t = s_in.c, s_in.F, s_in.d, s_in.H
    c, F, d, H = s_out.c, s_out.F, s_out.d, s_out.H
    r = 1.0 / O.gc_ratio(prm)
    Heff = H * r
    Hbar = float(np.mean(Heff))

    # ---- (F, H, d) block, transposed block Gauss-Seidel
    psi, Z, psi_c, psi_E = psi_terms(F, c, prm)
    chi = (psi > H_t).astype(float)
    Pd = stress_dd(F, c, d, prm)

    def solve_M(rhs):  # G K G lambda = G rhs, G the projection of mixed control if any
        lam, it = O.cg(lambda x: O.mech_apply(F, c, d, prm, x), O.apply_G_mixed(rhs, prm),
                       tol.tol_cg, tol.max_cg)
        if stats is not None:
            stats["cg_mech"] = stats.get("cg_mech", 0) + it
        return lam

    def solve_D(rhs):
        lam, it = O.pcg(lambda x: O.pff_apply(x, Heff, prm),
                        lambda q: O.pff_precond(q, Hbar, prm), rhs, tol.tol_pff_cg,
                        tol.max_cg, np.zeros_like(rhs))
        if stats is not None:
            stats["cg_pff"] = stats.get("cg_pff", 0) + it
        return lam

    def sweep(seedF, seedD, lamH):
        lamM = solve_M(seedF + chi * lamH * Z)
        return lamM, solve_D(seedD - O.ddot(Pd, lamM))

    # lamD = lamD0 + T lamD with T x = sweep(0, 0, 2 r (1-d) x): one transposed
    # Gauss-Seidel sweep is lamD0, and GMRES solves (I - T) lamD = lamD0 (T has rank at most
    # the number of voxels on the active branch of the history)
    lamM, lamD = sweep(seeds["F"], seeds["d"], seeds["H"])
    if stats is not None:
        stats["sweeps"] = stats.get("sweeps", 0) + 1
    if chi.any():
        zF = np.zeros_like(seeds["F"])
        zD = np.zeros_like(seeds["d"])

        def IminusT(x):
            if stats is not None:
                stats["sweeps"] = stats.get("sweeps", 0) + 1
            return x - sweep(zF, zD, 2.0 * r * (1.0 - d) * x)[1]
        lamD, _ = gmres(IminusT, lamD, tol.tol_stag, tol.max_stag)
        lamM = solve_M(seeds["F"] + chi * (seeds["H"] + 2.0 * r * (1.0 - d) * lamD) * Z)
    lamH = seeds["H"] + 2.0 * r * (1.0 - d) * lamD

    P = O.stress(F, c, d, prm)
    gE = -O.ddot(lamM, P) + chi * lamH * psi_E
    gG = chi * lamH * psi - 2.0 * r * H * (1.0 - d) * lamD
    sH_t = (1.0 - chi) * lamH
    gc_tot = seeds["c"] - O.ddot(stress_dc(F, c, d, prm), lamM) + chi * lamH * psi_c

    # ---- chemistry: (I + dt M L)^T lam = gc_tot, M = dmu~/dc.  The chemistry sees
    # F~ = F_t + Fcmd - Fbar_t; under mixed control Fbar_t is mean(F_t) on the controlled
    # components, so there dF~/dF_t = I - mean and the seed of F_t loses its mean
    Ft = F_t + (s_out.Fcmd - s_in.Fbar).reshape(3, 3, 1, 1, 1)
    K = O.chem_conductivity(Ft, c_t, d_t, prm)
    mue, mue_F, mue_c = mu_elastic_derivs(Ft, c, d_t, prm)
    m = 1.0 / (c * (1.0 - c)) + mue_c / prm.RT
    if not np.all(m > 0.0):
        raise FloatingPointError("chemistry Jacobian not positive (dmu~/dc <= 0)")
    lamC, it = O.cg(lambda y: O.chem_apply(y, m, K, dt, prm), gc_tot / m, tol.tol_chem_cg,
                    tol.max_cg)
    if stats is not None:
        stats["cg_chem"] = stats.get("cg_chem", 0) + it
    mu = O.chem_potential(c, Ft, d_t, prm)
    gl = fd_gradient(lamC, prm)
    gm = fd_gradient(mu, prm)
    s = np.einsum("i...,ij...,j...->...", gl, K, gm)
    Ll = O.chem_L(lamC, K, prm)
    phi = O.mobility_phi(d_t)
    dphi = -1.8 * (1.0 - d_t) + 0.2 * d_t
    sc_t = lamC - dt * (1.0 - 2.0 * c_t) / (c_t * (1.0 - c_t)) * s
    sd_t = -dt * dphi / phi * s + dt * Ll * 2.0 * mue / ((1.0 - d_t) * prm.RT)
    sF_t = -dt * conductivity_form_dF(Ft, c_t, d_t, gl, gm, prm) - dt * Ll * mue_F / prm.RT
    if prm.stress_mask is not None and s_in.mean_controlled:
        M = np.asarray(prm.stress_mask, dtype=bool)
        sF_t[M] -= sF_t[M].mean(axis=(1, 2, 3), keepdims=True)
    gD = -dt * s
    gE = gE - dt * Ll * mue / prm.RT
    return dict(c=sc_t, F=sF_t, d=sd_t, H=sH_t), dict(E=gE, gc=gG, D=gD)


def adjoint(prm, traj, dts, seeds_final, tol, stats=None):
    """Reverse over the trajectory; returns dict(E, gc, D) of dL/dlog-parameters from the
    steps (add the loss's own direct terms) and the seeds of the initial state."""
    grads = dict(E=np.zeros(prm.shape), gc=np.zeros(prm.shape), D=np.zeros(prm.shape))
    seeds = {k: np.array(v, dtype=float) for k, v in seeds_final.items()}
    for n in range(len(dts), 0, -1):
        seeds, g = step_adjoint(prm, traj[n - 1], traj[n], dts[n - 1], seeds, tol, stats)
        for k in grads:
            grads[k] += g[k]
    return grads, seeds


def crack_energy_gradient(prm, c_init, cdot_B, dts, Fbars, tol, stats=None):
    """Gamma_E of the final phase field and its gradient with respect to the per-voxel
    log E, log g_c and log D.  Returns (value, dict(E, gc, D))."""
    traj = forward(prm, c_init, cdot_B, dts, Fbars, tol)
    val, seed_d, dens = crack_energy_seed(traj[-1].d, prm)
    z = np.zeros(prm.shape)
    grads, _ = adjoint(prm, traj, dts, dict(c=z, F=np.zeros((3, 3) + prm.shape), d=seed_d, H=z),
                       tol, stats)
    grads["gc"] = grads["gc"] + dens
    return val, grads
