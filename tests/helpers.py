"""Shared test helpers: oracle parameters from a workload, error measures, tolerances."""
import numpy as np

from oracle import fg_oracle as O

# Relative tolerances (max |gpu - oracle| / max |oracle|) of one operator application.
# FP64: a few ulps per radix stage.  FP32: about eps32 x (log2 V + pointwise terms).
TOL_APPLY_FP64 = 1e-12
TOL_APPLY_FP32 = 1e-5
# float-float transforms (pairs of FP32, about 48 significant bits) of FP64 fields
TOL_APPLY_FF = 1e-13
# FP64 coupled step against the oracle (the GPU FP64 bar)
TOL_STEP_FP64 = 1e-10


def oracle_params(w_or_phases, phase_id=None, h=None, gc=1.0, lc=2e-7, RT=8.314462618 * 298.15,
                  cmax=3.0e4):
    if phase_id is None:
        w = w_or_phases
        return O.make_params([O.Phase(**vars(p)) for p in w.phases], w.phase_id, w.h, gc=w.gc,
                             lc=w.lc, RT=w.RT, cmax=w.cmax, log_E=w.log_E, log_D=w.log_D,
                             log_gc=w.log_gc, log_smax=w.log_smax)
    return O.make_params([O.Phase(**vars(p)) for p in w_or_phases], phase_id, h, gc=gc, lc=lc,
                         RT=RT, cmax=cmax)


def rel_err(a, b):
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def homogeneous_stretch_damage(E, nu, smax, gc, lc, l):
    """History and phase field of a homogeneous compressible Neo-Hookean medium (no
    swelling) under F = diag(l, 1, 1): the Cauchy stress is diagonal, sigma_xx =
    (G (l^2 - 1) + lam ln l)/l and sigma_yy = sigma_zz = lam ln l / l, so D_f =
    sum (<sigma_i>/sigma_max)^2 - 1 (Eq. SigDrivingForce), H = g_c/(2 l_c) <D_f>, and the
    uniform solution of Eq. PFFA is d = 2H/(g_c/l_c + 2H).  Returns (H, d)."""
    import math
    lam, G = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    sx = (G * (l * l - 1.0) + lam * math.log(l)) / l
    sy = lam * math.log(l) / l
    Df = max((max(sx, 0.0) / smax) ** 2 + 2.0 * (max(sy, 0.0) / smax) ** 2 - 1.0, 0.0)
    Hx = gc / (2.0 * lc) * Df
    return Hx, 2.0 * Hx / (gc / lc + 2.0 * Hx)

