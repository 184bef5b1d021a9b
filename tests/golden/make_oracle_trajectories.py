"""Writes the oracle's coupled-step trajectories that the GPU tests compare against.

Each case runs the CPU oracle (``oracle/fg_oracle.py``, FP64) on a seeded workload from
``paper_2411_16583_gb300/synth.py`` for a number of coupled steps (Alg. 4) and stores, for
the recorded steps, the fields at a fixed sample of voxels together with whole-field
summaries.  Nothing here calls the CUDA path.  The runs take minutes to hours on one CPU
core, which is why their results are stored instead of recomputed in every GPU test run.

    python tests/golden/make_oracle_trajectories.py <case> [<case> ...]

Cases:
    ellipsoid32  the 128^3 rough-ellipsoid particle recipe at a quarter of its size
                 (32^3; semi-axes 12.5/10/8.75, roughness std 0.375 / correlation 1,
                 band 2, 50-step influx), run until the first step with damage and two
                 steps beyond it (at most 50 steps)
    plate        the Sec. 4.3 plate (64 x 64 x 1, Saint-Venant-Kirchhoff, Omega = 1.3) at
                 Newton and staggered tolerance 1e-12, until the first damaging step (at
                 most 20; the step after it takes the oracle over an hour at 1e-12)
    gumbel512    the Sec. 5.1 disc (512^2, Saint-Venant-Kirchhoff, Gumbel-distributed
                 stiffness and strength, Omega = 1.3, full chemistry Jacobian): its first
                 two steps (the second one damages)

Recorded steps: the last undamaged step, the first damaging step and the steps after it
that the case asks for (or the last step when nothing cracks).  Output
``tests/golden/<case>.npz`` holds, per recorded step s (arrays suffixed _s<k>):
the flat voxel indices of the sample (a seeded random set plus the voxels of largest d),
F (9 x n), c, d, H at those voxels, and the scalars mass = sum c, the fracture energy of
Eq. crack, max d, the number of voxels with d > 1e-3 and the staggered iterations.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import fg_oracle as O  # noqa: E402
from paper_2411_16583_gb300 import synth as S  # noqa: E402

N_RANDOM = 1536   # seeded random sample voxels
N_DAMAGED = 128   # plus the voxels of largest d at the recorded step


def workload(case):
    """The seeded workload of a case (also used by the GPU tests)."""
    if case == "ellipsoid32":
        f = 32 / 128
        return S.ellipsoid(n=32, axes=(50 * f, 40 * f, 35 * f), rough_std=1.5 * f,
                           rough_corr=4 * f, band=2, nsteps=50)
    if case == "plate":
        # Newton 1e-12: with the paper's buffer at 1e-5 of the plate's stiffness the fields
        # are fixed only to the solver tolerance times a large condition number, so the
        # comparison runs well below the default 1e-9
        w = S.plate()
        w.tol = dict(w.tol, tol_newton=1e-12, tol_stag=1e-12, tol_cg=1e-13, tol_chem=1e-12,
                     tol_chem_cg=1e-13, tol_pff_cg=1e-13)
        return w
    if case == "gumbel512":
        return S.gumbel_disc()
    raise ValueError(case)


MAX_STEPS = {"ellipsoid32": 50, "plate": 20, "gumbel512": 2}
AFTER_DAMAGE = {"ellipsoid32": 2, "plate": 0, "gumbel512": 0}


def oracle_params(w):
    return O.make_params([O.Phase(**vars(p)) for p in w.phases], w.phase_id, w.h, gc=w.gc,
                         lc=w.lc, RT=w.RT, cmax=w.cmax, log_E=w.log_E, log_D=w.log_D,
                         log_gc=w.log_gc, log_smax=w.log_smax)


def sample(st, V, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = rng.choice(V, size=min(N_RANDOM, V), replace=False)
    top = np.argsort(st.d.ravel())[-N_DAMAGED:]
    return np.unique(np.concatenate([idx, top]))


def record(k, st, prm, stats, V):
    idx = sample(st, V, 1000 + k)
    return {f"idx_s{k}": idx,
            f"F_s{k}": st.F.reshape(9, V)[:, idx],
            f"c_s{k}": st.c.ravel()[idx],
            f"d_s{k}": st.d.ravel()[idx],
            f"H_s{k}": st.H.ravel()[idx],
            f"scal_s{k}": np.array([st.c.sum(), O.crack_energy(st.d, prm), st.d.max(),
                                    float((st.d > 1e-3).sum()), float(stats["stag"])])}


def run(case):
    w = workload(case)
    prm = oracle_params(w)
    V = w.nvox
    st = O.CoupledState(prm, w.c_init, w.cdot_B, O.Tolerances(**w.tol))
    out = {}
    recorded = []
    first_damage = None
    prev = None  # the record of the step before (kept until damage appears)
    log = open(os.path.join(HERE, f"{case}.log"), "w")
    for k in range(1, MAX_STEPS[case] + 1):
        t0 = time.time()
        stats = st.step(w.dt, np.eye(3))
        nd = int((st.d > 1e-3).sum())
        log.write(json.dumps({"step": k, "s": round(time.time() - t0, 1), "stag": stats["stag"],
                              "cg_mech": stats.get("cg_mech", 0), "cg_pff": stats.get("cg_pff", 0),
                              "dmax": float(st.d.max()), "damaged": nd}) + "\n")
        log.flush()
        rec = record(k, st, prm, stats, V)
        if first_damage is None and nd > 0:
            first_damage = k
            if prev is not None:  # the last undamaged step as well
                out.update(prev)
                recorded.append(k - 1)
        if first_damage is not None or k == MAX_STEPS[case]:
            out.update(rec)
            recorded.append(k)
        prev = rec
        if first_damage is not None and k >= first_damage + AFTER_DAMAGE[case]:
            break
    out["steps"] = np.array(recorded)
    out["first_damage"] = np.array(first_damage if first_damage is not None else -1)
    np.savez_compressed(os.path.join(HERE, f"{case}.npz"), **out)
    log.close()


if __name__ == "__main__":
    for case in sys.argv[1:]:
        run(case)
