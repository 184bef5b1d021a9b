"""Benchmark: coupled time steps of the FFT chemo-mechanical fracture method on GB300.

Default workload: the 256^3 rough ellipsoidal particle (semi-axes 100/80/70 voxels,
roughness std 3 / correlation 8, influx band 8 voxels, smooth Gaussian concentration
perturbation of std 0.02), mixed FP32/FP64 precision, Newton tolerance 1e-9.  One bench
step is one coupled time step (Alg. 4: chemistry Newton-CG, then the staggered mechanics
Newton-CG and phase-field PCG) through the C ABI, every part of it in the CUDA library.
Inputs are resident on the device when the timed region starts; the working set
(~15 GB) is far larger than L2 (129 MB), so nothing stays cached between steps.

Rank 0 prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("coupled time-step wall time & fused-matvec voxel-applies/s at 256³, "
          "mixed vs FP64")
UNIT = "voxel-steps/s"

# Algorithmic bytes per voxel of each profiled launch site of the FP32 mechanical CG
# iteration (9-component fields, 4-byte reals; the half spectrum holds (nx/2+1)/nx of a
# real field as complex numbers, so a 9-component spectrum is 72 (nx/2+1)/nx B/voxel).
# DRAM bytes per voxel that ncu measured per launch of the fused CG X passes (dram bytes
# read + written on a 256 x 256 x 64 grid, divided by its voxels; x rows of 256): valid for
# these kernels as they are, at nx = 256
MEASURED_TRAFFIC_B_PER_VOXEL = {"xi": 203.6, "xf": 181.2}


# algorithmic minimum of one FP32 mechanical operator application, per voxel:
# read x (9 x 4 B) and the state (F 9 x 4 B, c, d, phase), write y (9 x 4 B)
MECH_ALG_B_PER_VOXEL = 116.0
# DRAM bytes per voxel that ncu measured over the five kernels of one FP32 mechanical
# operator application (fg_time_apply) on a 256 x 256 x 64 grid (x rows of 256), summed over
# the kernels and divided by the voxels (the autotuner's choices: no L2 prefetch, one
# column per block in the projection pass); valid for these kernels as they are
MEASURED_APPLY_TRAFFIC_B_PER_VOXEL = 386.5


def APPLY_SCHEDULED_B_PER_VOXEL(nx, clustered=False):
    """Bytes per voxel the passes of one FP32 operator application schedule: X-fwd reads x
    and the packed 12-real state and writes the half spectrum, Y-fwd, Z and Y-inv read and
    write it (the clustered Y-Z-Y pass once for all three), X-inv reads it and writes y (its
    <x, y> reads x once more)."""
    spec = 72.0 * (nx // 2 + 1) / nx
    return (36 + 48 + spec) + (1 if clustered else 3) * (2 * spec) + (spec + 36 + 36)


def _apply_traffic(nx, V):
    if MEASURED_APPLY_TRAFFIC_B_PER_VOXEL is None or nx != 256:
        return None
    return MEASURED_APPLY_TRAFFIC_B_PER_VOXEL * V


def site_bytes(nx):
    spec = 72.0 * (nx // 2 + 1) / nx
    return {0: 36 + 36 + 48 + 36 + spec,   # X-fwd: read r, p, tangent state; write p, spectrum
            1: 2 * spec,                    # Y-fwd: read + write spectrum
            2: 2 * spec,                    # Z + projection: read + write spectrum
            3: 2 * spec,                    # Y-inv: read + write spectrum
            4: spec + 3 * 36 + 2 * 36}      # X-inv: read spectrum, r, x, p; write r, x


SITE_NAMES = {0: "mech X-fwd: p = r + beta p, tangent, <p,Kp> (pass_kernel<XFwd<float,N,PCgTangentNH>>)",
              1: "mech Y-fwd (pass_kernel<YPassD<float,N,false>>, register-direct for N = 16^2)",
              2: "mech Z + projection (pass_kernel<ZPassD<float,N,ZProject>>)",
              3: "mech Y-inv (pass_kernel<YPassD<float,N,true>>)",
              4: "mech X-inv: r -= alpha q, x += alpha p, |r|^2 (pass_kernel<XInv<float,N,ECgUpdate1,true>> per component, or ECgUpdate)"}


def _traffic(site, nx, voxels_per_launch):
    """Measured DRAM bytes per launch of the dominant site (None without a capture)."""
    key = {4: "xi", 0: "xf"}.get(site)
    if key is None or nx != 256:
        return None
    return MEASURED_TRAFFIC_B_PER_VOXEL[key] * voxels_per_launch


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (the slowest rank sets the job's time); x itself when
    there is one rank (dist None)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(voxels_per_rank, world, seconds_per_step):
    """Whole-job voxel-steps/s: every rank advances its own RVE by one step."""
    return voxels_per_rank * world / seconds_per_step


# untimed steps before the warm-up: the timed window (after 5 warm-up steps, 20 timed) then
# covers steps 51-70 of the 100-step schedule, whose step times sit at the median of steps
# 11-100 (measured on a GB300: 987 ms, rising from 850 ms at step 11 to 1140 ms at step
# 100 as the Krylov counts grow).  The particle does not crack within the 100 steps (max d
# stays 0), so the phase-field solve is timed on the damaging Sec. 5.1 disc instead
START_STEPS = 45


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=256, help="grid edge of the particle workload")
    p.add_argument("--nz", type=int, default=0, help="override the z extent (profiling cases)")
    p.add_argument("--ny", type=int, default=0, help="override the y extent (profiling cases)")
    p.add_argument("--start", type=int, default=START_STEPS,
                   help="untimed steps before the warm-up (the timed window's position in the "
                        "100-step schedule)")
    p.add_argument("--site-steps", type=int, default=2,
                   help="steps of the separate per-kernel profiling pass")
    p.add_argument("--fp64-steps", type=int, default=1,
                   help="FP64 comparison from the window's first state (0: skip)")
    p.add_argument("--adjoint-steps", type=int, default=2,
                   help="taped steps of the 128^3 adjoint timing added to the line (0: skip)")
    p.add_argument("--batch-rves", type=int, default=64,
                   help="RVEs of the batch timing added to the line (0: skip)")
    p.add_argument("--damage-steps", type=int, default=3,
                   help="damaging steps of the 512^2 Sec. 5.1 disc timed for the line (0: skip)")
    p.add_argument("--trajectory-error", type=int, default=0,
                   help="only run this many steps of the workload in the mixed form and then in "
                        "the FP64 form, and print the per-field error of the mixed trajectory "
                        "against the FP64 one every quarter of the run (about 0.4 min + 21 s "
                        "per step at 256^3)")
    p.add_argument("--profile-apply", type=int, default=0,
                   help="only run this many FP32 mechanical operator applications on the "
                        "workload (a small case for ncu captures) and print their time")
    p.add_argument("--l2-prefetch", type=int, default=0,
                   help="profile-apply: the X passes' L2 prefetch (the autotuner's choice)")
    p.add_argument("--z-columns", type=int, default=0,
                   help="profile-apply: columns per block of the projection pass (0, 1, 4)")
    p.add_argument("--cluster-pass", type=int, default=1,
                   help="profile-apply: the clustered Y-Z-Y pass where it applies (1) or the "
                        "three separate passes (0)")
    p.add_argument("--cpu-seconds", type=float, default=20.0, help="oracle sample budget")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--adjoint", action="store_true",
                   help="time the coupled adjoint (128^3 ellipsoid with log fields, FP64, "
                        "checkpoints every 5 steps) instead of the step benchmark")
    p.add_argument("--batch", type=int, default=0,
                   help="batched RVEs: N particles of seeded sizes {48,64,80,96}^3 (0: off)")
    return p.parse_args()


def workload_desc(a):
    """The timed workload, the same words for both arms."""
    first = a.start + a.warmup + 1
    return (f"rough ellipsoid particle {a.n}^3, coupled steps of Alg. 4 at Newton tolerance "
            f"1e-9; buffer E x 1e-2 of the particle's; smooth Gaussian concentration field of "
            f"std 0.02 around c = 0.07 inside the particle, whose stress-free c0 is 0.07; "
            f"100-step influx schedule, timed steps {first}-{first + a.steps - 1} after "
            f"{a.start} untimed steps and {a.warmup} warm-up steps")


def _workload(n, seed, nz=0, ny=0):
    from paper_2411_16583_gb300 import synth as S
    if n == 256 and not nz and not ny:
        return S.ellipsoid256(seed=seed)
    f = n / 256.0
    shape = (nz or n, ny or n, n) if (nz or ny) else None
    axes = (100 * f, min(80 * f, 0.4 * ny) if ny else 80 * f,
            min(70 * f, 0.4 * nz) if nz else 70 * f)
    return S.ellipsoid(n=n, axes=axes, rough_std=3 * f, rough_corr=8 * f,
                       band=max(1, round(8 * f)), nsteps=100, seed=seed, c_perturb=0.02,
                       shape=shape, phases=S.default_phases(buffer_E=S.BENCH_BUFFER_E))


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if r and num(r[0]) is not None]
        mx = [num(r[1]) for r in self.rows if len(r) > 1 and num(r[1]) is not None]
        pw = [num(r[2]) for r in self.rows if len(r) > 2 and num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# Per-step operator counts used to express the oracle's per-operator times in the
# metric's unit when no GPU step is available (the --impl reference arm): the counts of
# the FP64 form's step 51 of this workload (the first step of the timed window), whose
# Krylov iterations follow the oracle's (measured on a GB300).
DEFAULT_STEP_PROFILE = {"cg_mech": 461, "newton_mech": 2, "stag": 1, "cg_chem": 695,
                        "newton_chem": 9, "cg_pff": 0}


def oracle_step_seconds(w, budget_s, profile, reuse=None):
    """Times the oracle's operators on the full-size fields of workload w (a bounded
    sample, about budget_s seconds) and combines them with the operator counts of one
    coupled step.  reuse (dict op -> seconds) supplies earlier timings of operators that
    are not timed again.  Returns (seconds per step, description of the sample, the
    per-operator seconds)."""
    import numpy as np
    from oracle import fg_oracle as O
    from paper_2411_16583_gb300 import synth as S
    prm = O.make_params([O.Phase(**vars(p)) for p in w.phases], w.phase_id, w.h, gc=w.gc,
                        lc=w.lc, RT=w.RT, cmax=w.cmax)
    F, c, d = S.random_state(w.shape, seed=1, f_amp=0.01, c_lo=0.01, c_hi=0.3, d_hi=0.0)
    x = S.random_tensor_field(w.shape, 2).reshape((3, 3) + w.shape)
    y = S.random_tensor_field(w.shape, 3, ncomp=1)[0]
    Kc = O.chem_conductivity(F, c, d, prm)
    m = 1.0 / (c * (1.0 - c))
    ops = {"mech": lambda: O.mech_apply(F, c, d, prm, x),
           "gres": lambda: O.apply_G(x, prm.h),
           "chem": lambda: O.chem_apply(y, m, Kc, 1.0, prm)}
    times, counts = dict(reuse or {}), {k: 0 for k in (reuse or {})}
    t_start = time.perf_counter()
    share = budget_s / len(ops)
    for k, f in ops.items():
        if reuse and k in reuse:
            continue
        n, t0 = 0, time.perf_counter()
        while True:
            f()
            n += 1
            if time.perf_counter() - t0 > share:
                break
        times[k] = (time.perf_counter() - t0) / n
        counts[k] = n
    p = profile
    # a Newton iteration applies the residual projection once (twice in mixed mode, which
    # also projects the correction); each staggered check applies it twice (residual and
    # its normalisation); each chemistry Newton iteration evaluates its residual with one
    # operator-equivalent round trip
    step = (p["cg_mech"] * times["mech"]
            + (p["newton_mech"] + 1 + 2 * (p["stag"] + 1)) * times["gres"]
            + (p["cg_chem"] + p["newton_chem"]) * times["chem"])
    desc = (f"oracle operators on the full {w.shape[2]}^3 fields: "
            + ", ".join(f"{counts[k]} x {k} ({times[k]:.2f} s each)" for k in ops)
            + f", combined with one step's operator counts {p}; "
            + f"{time.perf_counter() - t_start:.0f} s of CPU work")
    return step, desc, times


def _cores():
    try:
        import numpy as np  # noqa: F401
        return int(os.environ.get("OMP_NUM_THREADS") or 1)
    except Exception:
        return 1


def cufft_comparator(sol, w, device="cuda", reps=10):
    """The same FP32 mechanical operator built from cuFFT's batched 3D real transforms over
    the nine components and two separate element-wise kernels (tangent, projection),
    libfg_cufft.so: the timed library comparator of the fused apply.  Returns (ms per
    apply, max |y - y_fused| / max |y_fused|)."""
    import ctypes as C
    import numpy as np
    import torch
    from paper_2411_16583_gb300 import binding as B, build
    lib = C.CDLL(build.build_comparator())
    lib.fgc_last_error.restype = C.c_char_p
    V = w.nvox
    nz, ny, nx = w.shape
    pid = w.phase_id.ravel()
    tab = lambda attr: np.array([getattr(p, attr) for p in w.phases])[pid]
    E = tab("E") * (np.exp(w.log_E.ravel()) if w.log_E is not None else 1.0)
    nu = tab("nu")
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)
    F = sol.get(B.FIELD_F, device=device)
    c = sol.get(B.FIELD_C, device=device)
    d = sol.get(B.FIELD_D, device=device)
    L, M, Om, c0 = dev(lam), dev(mu), dev(tab("Omega")), dev(tab("c0"))
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn(9 * V, dtype=torch.float32, generator=g).to(device)
    y = torch.empty_like(x)
    yf = torch.empty_like(x)
    sol.apply(B.OP_MECH, x, yf, prec=1)
    ms = C.c_float()
    torch.cuda.synchronize()
    P = lambda t: C.c_void_p(t.data_ptr())
    rc = lib.fgc_mech_apply(nx, ny, nz, C.c_double(w.h[0]), C.c_double(w.h[1]),
                            C.c_double(w.h[2]), P(F), P(c), P(d), P(L), P(M), P(Om), P(c0),
                            P(x), P(y), reps, C.byref(ms),
                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise RuntimeError(lib.fgc_last_error().decode())
    diff = float((y - yf).abs().max() / yf.abs().max())
    return float(ms.value), diff


def crack_energy(d, w):
    """Fracture energy sum g_c (d^2/(2 l_c) + l_c/2 |grad_f d|^2) h^3 (Eq. crack) of a CUDA
    tensor d (nz, ny, nx), forward differences with periodic wrap; a reported figure."""
    import torch
    g2 = torch.zeros_like(d)
    for axis, h in ((2, w.h[0]), (1, w.h[1]), (0, w.h[2])):
        if d.shape[axis] > 1:
            g2 += ((torch.roll(d, -1, axis) - d) / h) ** 2
    dens = w.gc * (d * d / (2 * w.lc) + 0.5 * w.lc * g2)
    return float(dens.sum()) * w.h[0] * w.h[1] * w.h[2]


def _state(sol):
    """Device copies of the evolving state (F, c, d, H)."""
    from paper_2411_16583_gb300 import binding as B
    return {f: sol.get(f, device="cuda") for f in (B.FIELD_F, B.FIELD_C, B.FIELD_D, B.FIELD_H)}


def _restore(sol, st):
    for f, t in st.items():
        sol.set(f, t)


def _timed_step(sol, w, stream):
    """One coupled step timed with CUDA events on the context's stream: (ms, stats)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = sol.step(w.dt)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), st


def fp64_split(w, sol, state0, stream):
    """From one saved state of the mixed run: a mixed step, an FP64 step at the FP64
    form's Krylov tolerance and an FP64 step at the mixed form's inner (forcing) tolerance.
    Reports the three times and Krylov counts, and the mixed step's per-field error against
    the FP64 step (max |dF| / max |F|, the same for c, max |dd|, and the fracture energy's
    relative error)."""
    from paper_2411_16583_gb300 import binding as B
    out = {}
    _restore(sol, state0)
    ms_m, st_m = _timed_step(sol, w, stream)
    mixed = _state(sol)
    forcing = sol.opts.cg_forcing
    # the mixed form with its residual transforms in FP64 arithmetic instead of float-float
    m64 = B.from_workload(w, precision=B.FG_MIXED, stream=stream.cuda_stream, residual_ff=0)
    _restore(m64, state0)
    ms_m64, st_m64 = _timed_step(m64, w, stream)
    mixed64 = _state(m64)
    m64.close()
    runs = {"fp64": {}, "fp64_at_forcing": {"tol_cg": forcing, "tol_chem_cg": forcing}}
    ref = None
    for name, kw in runs.items():
        s64 = B.from_workload(w, precision=B.FG_FP64, stream=stream.cuda_stream, **kw)
        _restore(s64, state0)
        ms, st = _timed_step(s64, w, stream)
        out[name] = {"ms": ms, "stats": st}
        if name == "fp64":
            ref = _state(s64)
        s64.close()
    out["mixed"] = {"ms": ms_m, "stats": st_m,
                    "residual_transforms": "float-float" if sol.opts.residual_ff else "FP64"}
    out["mixed_fp64_residuals"] = {"ms": ms_m64, "stats": st_m64}
    rel = lambda a, b: float((a - b).abs().max() / b.abs().max())
    out["mixed_fp64_residuals"]["vs_fp64_error"] = {
        "F_max_rel": rel(mixed64[B.FIELD_F], ref[B.FIELD_F]),
        "c_max_rel": rel(mixed64[B.FIELD_C], ref[B.FIELD_C])}
    gm, gr = crack_energy(mixed[B.FIELD_D], w), crack_energy(ref[B.FIELD_D], w)
    out["mixed_vs_fp64_error"] = {
        "F_max_rel": rel(mixed[B.FIELD_F], ref[B.FIELD_F]),
        "c_max_rel": rel(mixed[B.FIELD_C], ref[B.FIELD_C]),
        "d_max_abs": float((mixed[B.FIELD_D] - ref[B.FIELD_D]).abs().max()),
        "crack_energy_rel": abs(gm - gr) / gr if gr > 0 else None,
        "crack_energy_fp64": gr,
        "bars": {"F_max_rel": 1e-7, "c_max_rel": 1e-7, "d_max_abs": 1e-6, "crack_energy_rel": 1e-6}}
    out["precision_speedup"] = out["fp64_at_forcing"]["ms"] / ms_m
    out["krylov_speedup"] = out["fp64"]["ms"] / out["fp64_at_forcing"]["ms"]
    return out


def _oracle_worker(args):
    n, budget, counts = args
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    w = _workload(n, 0)
    return oracle_step_seconds(w, budget, counts)[0]


def oracle_all_cores(n, budget_s, counts):
    """The oracle's operator sample on every host core at once: one process per core (spawn,
    one BLAS thread each), each timing the same sample on its own copy of the n^3 fields
    with the given per-step operator counts.  Returns (voxel-steps/s of all processes
    together, processes)."""
    import multiprocessing as mp
    procs = max(1, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        secs = pool.map(_oracle_worker, [(n, budget_s, counts)] * procs)
    return sum(n ** 3 / s for s in secs), procs


def main():
    a = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return reference_arm(a, rank, world)
    if a.batch:
        print(json.dumps(batch_mode(a.batch, a.steps, a.warmup)))
        return
    if a.adjoint:
        print(json.dumps(adjoint_mode(a.n if a.n != 256 else 128, a.steps, a.warmup)))
        return
    if a.profile_apply:
        print(json.dumps(profile_apply(a)))
        return
    if a.trajectory_error:
        print(json.dumps(trajectory_error(a)))
        return
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()  # a capturable stream: the CG's CUDA graphs replay on it
    with torch.cuda.stream(stream):
        line = run_ours(a, rank, world, local, dist, stream)
    if rank == 0:
        print(json.dumps(line))


def run_ours(a, rank, world, local, dist, stream):
    import torch
    from paper_2411_16583_gb300 import binding as B
    w = _workload(a.n, seed=rank, nz=a.nz)
    sol = B.from_workload(w, precision=B.FG_MIXED, stream=stream.cuda_stream)
    V = w.nvox
    tuned_ms = sol.autotune()
    tuning = sol.autotune_report()
    for _ in range(a.start):  # advance to the measured window (untimed)
        sol.step(w.dt)
    for _ in range(a.warmup):
        sol.step(w.dt)
    state0 = _state(sol) if (a.fp64_steps > 0 and rank == 0) else None

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    stats, step_ms = [], []
    with Clocks(local) as clk:
        barrier()
        l0 = B.kernel_launches()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
        ev[0].record(stream)
        for k in range(a.steps):
            stats.append(sol.step(w.dt))
            ev[k + 1].record(stream)
        barrier()
        launches = B.kernel_launches() - l0
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(a.steps)]
    ms = max_over_ranks(ev[0].elapsed_time(ev[-1]) / a.steps, dist, "cuda")
    d_end = sol.get(B.FIELD_D, device="cuda")
    window = {"first_step": a.start + a.warmup + 1, "last_step": a.start + a.warmup + a.steps,
              "median_step_ms": statistics.median(step_ms), "min_step_ms": min(step_ms),
              "max_step_ms": max(step_ms),
              "steps_with_phase_field_cg": sum(1 for s in stats if s["cg_pff"] > 0),
              "damaged_voxels_at_end": int((d_end > 1e-3).sum()), "d_max_at_end": float(d_end.max()),
              "cg_graph_replays": sum(s["cg_graph_replays"] for s in stats),
              "totals": {k: sum(s[k] for s in stats) for k in
                         ("newton_chem", "newton_mech", "cg_chem", "cg_mech", "cg_pff", "stag")}}
    del d_end

    # per-site kernel times of the mechanical CG in a separate pass (CUDA events around
    # every launch of a site; graphs do not replay while a site is profiled)
    for s in range(5):
        sol.profile(s, True)
    for _ in range(a.site_steps):
        sol.step(w.dt)
    prof = {s: sol.profile_read(s) for s in range(5)}
    for s in range(5):
        sol.profile(s, False)

    # end to end through the same public calls with host buffers: each step copies the
    # state (F, c, d, H) in from pinned host memory and the new (F, c, d) back out
    e2e = None
    if not a.no_e2e:
        hF = torch.empty(9 * V, dtype=torch.float64).pin_memory()
        hs = [torch.empty(V, dtype=torch.float64).pin_memory() for _ in range(3)]
        lib = sol.lib
        for f, buf in ((B.FIELD_F, hF), (B.FIELD_C, hs[0]), (B.FIELD_D, hs[1]), (B.FIELD_H, hs[2])):
            sol._check(lib.fg_get_field(sol.ctx, f, B._ptr(buf), 0))
        barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            for f, buf in ((B.FIELD_F, hF), (B.FIELD_C, hs[0]), (B.FIELD_D, hs[1]),
                           (B.FIELD_H, hs[2])):
                sol._check(lib.fg_set_field(sol.ctx, f, B._ptr(buf), 0))
            sol.step(w.dt)
            for f, buf in ((B.FIELD_F, hF), (B.FIELD_C, hs[0]), (B.FIELD_D, hs[1])):
                sol._check(lib.fg_get_field(sol.ctx, f, B._ptr(buf), 0))
        barrier()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / a.steps, dist, "cuda")
        e2e = {"value": job_throughput(V, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": 12 * V * 8,
               "d2h_bytes_per_step": 11 * V * 8}

    # fused matvec rates (50 applications after 5 warm-ups, CUDA events):
    # the FP32 operators of the mixed context, and the cuFFT comparator of the mechanical one
    sol.time_apply(B.OP_MECH, 1, 5)
    mech32_ms = sol.time_apply(B.OP_MECH, 1, 50)
    matvec = {"mech_fp32_ms": mech32_ms, "mech_fp32_voxel_applies_per_s": V / (mech32_ms * 1e-3)}
    for name, op, prec in (("pff_fp32", B.OP_PFF, 1), ("pff_prec_fp32", B.OP_PFF_PREC, 1),
                           ("chem_fp32", B.OP_CHEM, 1), ("gres_fp64", B.OP_GRES, 0),
                           ("gres_float_float", B.OP_GRES, 2)):
        t = sol.time_apply(op, prec, 20)
        matvec[name + "_ms"] = t
        matvec[name + "_voxel_applies_per_s"] = V / (t * 1e-3)
    if rank == 0:
        try:
            cms, cdiff = cufft_comparator(sol, w)
            matvec["cufft_comparator"] = {
                "kind": "cuFFT batched 3D R2C/C2R over the nine components (cufftPlanMany) + "
                        "separate tangent and projection kernels, FP32",
                "ms_per_apply": cms, "voxel_applies_per_s": V / (cms * 1e-3),
                "max_rel_diff_vs_fused": cdiff, "fused_speedup": cms / mech32_ms}
        except Exception as e:  # noqa: BLE001
            matvec["cufft_comparator"] = {"unavailable": str(e)[:200]}
    out = {}
    if state0 is not None:
        out["fp64_split"] = fp64_split(w, sol, state0, stream)
        out["fp64_step_ms"] = out["fp64_split"]["fp64"]["ms"]
        del state0
    sol.close()
    if rank != 0:
        return None
    if a.fp64_steps > 0:
        s64 = B.from_workload(w, precision=B.FG_FP64, stream=stream.cuda_stream)
        s64.time_apply(B.OP_MECH, 0, 2)
        t64 = s64.time_apply(B.OP_MECH, 0, 10)
        matvec["mech_fp64_ms"] = t64
        matvec["mech_fp64_voxel_applies_per_s"] = V / (t64 * 1e-3)
        s64.close()
    peaks, src = _peaks()
    sb = site_bytes(w.shape[2])
    sites = {}
    names = dict(SITE_NAMES)
    if tuning.get("cluster_yzy_mech"):
        names[2] = ("mech Y-fwd + Z + projection + Y-inv in one clustered pass "
                    "(cluster_kernel<YZYCluster<float,N,ZRows>>, 16-CTA clusters)")
    for s, (n, t, vol) in prof.items():
        if n:
            sites[names[s]] = {"launches": n, "total_ms": t, "volumes": vol,
                                    "us_per_volume": t * 1e3 / vol,
                                    "alg_bytes_per_voxel": sb[s],
                                    "gbs": sb[s] * V * vol / (t * 1e-3) / 1e9,
                                    "frac_of_peak": sb[s] * V * vol / (t * 1e-3) / 1e9 / peaks["hbm_gbs"]}
    # the roofline: one fused mechanical operator application (five
    # pass kernels) moves at least 116 B per voxel (read x and the state, write y)
    ach = MECH_ALG_B_PER_VOXEL * V / (mech32_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC,
        "value": job_throughput(V, world, ms * 1e-3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_desc(a),
                   "precision": "mixed: FP32 Krylov operators, FP64 fields, residuals, norms "
                                "and updates (residual transforms in float-float arithmetic)",
                   "voxels": V, "l2": "inputs larger than L2 (no flush)",
                   "stream": "non-default (CUDA-graph replays on), profiling off"},
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": {"bound": "hbm",
                     "kernel": ("fused FP32 mechanical operator application (three pass "
                                "kernels: X-fwd tangent + R2C, clustered Y-Z-Y with the "
                                "projection, C2R X-inv)" if tuning.get("cluster_yzy_mech") else
                                "fused FP32 mechanical operator application (five pass "
                                "kernels: X-fwd tangent + R2C, Y-fwd, Z + projection, Y-inv, "
                                "C2R X-inv)"),
                     "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": ach / peaks["hbm_gbs"], "peak_source": src,
                     "alg_bytes_per_launch": MECH_ALG_B_PER_VOXEL * V,
                     "avg_launch_us": mech32_ms * 1e3,
                     "traffic": (None if tuning.get("cluster_yzy_mech") else
                                 _apply_traffic(w.shape[2], V)),
                     "scheduled_bytes_per_voxel": APPLY_SCHEDULED_B_PER_VOXEL(
                         w.shape[2], tuning.get("cluster_yzy_mech"))},
        "window": window,
        "kernels": sites,
        "matvec": matvec,
        "step_stats": stats[-1],
        "autotuned_apply_ms": tuned_ms,
        "autotune": tuning,
        "clocks": clk.summary(),
    }
    line.update(out)
    if a.adjoint_steps > 0:
        try:
            line["adjoint"] = adjoint_mode(128, a.adjoint_steps, 1)
        except Exception as e:  # noqa: BLE001
            line["adjoint"] = {"unavailable": str(e)[:200]}
    if a.damage_steps > 0:
        try:
            line["damaging"] = damaging_window(a.damage_steps)
        except Exception as e:  # noqa: BLE001
            line["damaging"] = {"unavailable": str(e)[:200]}
    if a.batch_rves > 0:
        try:
            line["batch"] = batch_mode(a.batch_rves, 2, 1)
        except Exception as e:  # noqa: BLE001
            line["batch"] = {"unavailable": str(e)[:200]}
    if not a.no_cpu_baseline:
        # the oracle is an FP64 method: its step takes the FP64 form's operator counts (of
        # this run when it timed an FP64 step, else those recorded at 256^3)
        counts = out.get("fp64_split", {}).get("fp64", {}).get("stats") or DEFAULT_STEP_PROFILE
        prof_counts = {k: counts[k] for k in DEFAULT_STEP_PROFILE}
        secs, desc, _ = oracle_step_seconds(w, a.cpu_seconds, prof_counts)
        line["cpu_baseline"] = {"value": V / secs, "unit": UNIT, "cores": 1,
                                "kind": "oracle", "sample": desc}
        try:
            allv, procs = oracle_all_cores(128, a.cpu_seconds / 2, prof_counts)
            line["cpu_baseline_all_cores"] = {
                "value": allv, "unit": UNIT, "cores": procs,
                "kind": "oracle",
                "sample": f"{procs} processes, each timing the oracle's operator sample on "
                          f"128^3 fields with the recorded 256^3 step counts; voxel-steps/s "
                          f"summed over the processes"}
        except Exception as e:  # noqa: BLE001
            line["cpu_baseline_all_cores"] = {"unavailable": str(e)[:200]}
    return line


def profile_apply(a):
    """n FP32 mechanical operator applications (fg_time_apply) on the workload's state after
    set-up: the command that ncu captures of the five pass kernels run."""
    import torch
    from paper_2411_16583_gb300 import binding as B
    w = _workload(a.n, 0, nz=a.nz, ny=a.ny)
    stream = torch.cuda.Stream()
    sol = B.from_workload(w, precision=B.FG_MIXED, stream=stream.cuda_stream,
                          l2_prefetch=a.l2_prefetch, z_columns=a.z_columns,
                          cluster_pass=a.cluster_pass)
    ms = sol.time_apply(B.OP_MECH, 1, a.profile_apply)
    sol.close()
    return {"mode": "profile-apply", "shape": list(w.shape), "applies": a.profile_apply,
            "cluster_pass": a.cluster_pass, "ms_per_apply": ms}


def trajectory_error(a):
    """The workload's first n steps in the mixed form, then in the FP64 form (Newton 1e-9,
    FP64 Krylov 1e-10), both on a side stream; the mixed fields are kept on the device at
    every quarter of the run and compared with the FP64 fields at the same step: max |dF| /
    max |F|, the same for c, max |dd| and the fracture energy's relative error (the bars of
    the mixed form: 1e-7, 1e-7, 1e-6, 1e-6)."""
    import torch
    from paper_2411_16583_gb300 import binding as B
    n = a.trajectory_error
    marks = sorted({max(1, (n * q) // 4) for q in (1, 2, 3, 4)})
    w = _workload(a.n, 0, nz=a.nz)
    stream = torch.cuda.Stream()
    out = {"mode": "trajectory-error", "workload": f"rough ellipsoid particle {a.n}^3, "
           f"100-step schedule", "steps": n, "marks": marks, "errors": {}, "ms_per_step": {}}
    with torch.cuda.stream(stream):
        kept = {}
        for prec, name in ((B.FG_MIXED, "mixed"), (B.FG_FP64, "fp64")):
            sol = B.from_workload(w, precision=prec, stream=stream.cuda_stream)
            t = 0.0
            for k in range(1, n + 1):
                ms, st = _timed_step(sol, w, stream)
                t += ms
                if k in marks:
                    if name == "mixed":
                        kept[k] = _state(sol)
                    else:
                        ref = _state(sol)
                        mix = kept.pop(k)
                        rel = lambda x, y: float((x - y).abs().max() / y.abs().max())
                        gm, gr = crack_energy(mix[B.FIELD_D], w), crack_energy(ref[B.FIELD_D], w)
                        out["errors"][k] = {
                            "F_max_rel": rel(mix[B.FIELD_F], ref[B.FIELD_F]),
                            "c_max_rel": rel(mix[B.FIELD_C], ref[B.FIELD_C]),
                            "d_max_abs": float((mix[B.FIELD_D] - ref[B.FIELD_D]).abs().max()),
                            "d_max": float(ref[B.FIELD_D].max()),
                            "crack_energy_rel": abs(gm - gr) / gr if gr > 0 else None}
                        del mix, ref
            out["ms_per_step"][name] = t / n
            sol.close()
    return out


def damaging_window(steps):
    """The Sec. 5.1 disc (512^2 Saint-Venant-Kirchhoff, Gumbel-distributed stiffness and
    strength, Omega = 1.3, 200-step schedule), mixed precision on a side stream: its first
    step is undamaged, the next `steps` crack, so they time the phase-field solves (Alg. 2)
    and the staggered iterations (Alg. 4).  Returns per-step times and counts."""
    import torch
    from paper_2411_16583_gb300 import binding as B, synth as S
    w = S.gumbel_disc()
    stream = torch.cuda.current_stream()
    sol = B.from_workload(w, precision=B.FG_MIXED, stream=stream.cuda_stream)
    sol.step(w.dt)
    rows = []
    for k in range(steps):
        ms, st = _timed_step(sol, w, stream)
        d = sol.get(B.FIELD_D, device="cuda")
        rows.append({"step": k + 2, "ms": ms, "stag": st["stag"], "cg_pff": st["cg_pff"],
                     "cg_mech": st["cg_mech"], "cg_chem": st["cg_chem"],
                     "damaged_voxels": int((d > 1e-3).sum()), "d_max": float(d.max())})
    sol.close()
    return {"workload": "Sec. 5.1 disc 512^2 x 1 (Saint-Venant-Kirchhoff, Gumbel stiffness and "
                        "strength, Omega = 1.3, full chemistry Jacobian, 200-step schedule), "
                        "mixed precision", "voxels": w.nvox, "steps": rows,
            "ms_per_step": sum(r["ms"] for r in rows) / len(rows)}


def adjoint_mode(n, steps, warmup):
    """Forward steps with a tape, then the reverse pass for dL/dlog(E, g_c, D) of a loss
    with random seeds on the final state; both timed with CUDA events on the context's
    stream (FP64 throughout).  Returns a dict."""
    import numpy as np
    import torch
    from paper_2411_16583_gb300 import binding as B, synth as S
    w = S.with_log_fields(S.ellipsoid(n=n, axes=(50 * n / 128, 40 * n / 128, 35 * n / 128),
                                      rough_std=1.5 * n / 128, rough_corr=4 * n / 128,
                                      band=max(1, round(8 * n / 128)), nsteps=50,
                                      phases=S.default_phases(buffer_E=S.BENCH_BUFFER_E)),
                          std=0.1)
    stream = torch.cuda.current_stream()
    sol = B.from_workload(w, precision=B.FG_FP64, stream=stream.cuda_stream)
    for _ in range(warmup):
        sol.step(w.dt)
    sol.tape(5)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record(stream)
    for _ in range(steps):
        sol.step(w.dt)
    e[1].record(stream)
    # a loss with seeded random dL/d(c, F, d) on the final state: every adjoint solve
    # runs (the fracture energy is zero until damage starts)
    rng = np.random.default_rng(0)
    dev = lambda a: torch.from_numpy(a).cuda()
    val, g, st = sol.adjoint(B.FG_LOSS_SEEDS, seed_c=dev(rng.standard_normal(w.shape)),
                             seed_F=dev(rng.standard_normal((3, 3) + w.shape)),
                             seed_d=dev(rng.standard_normal(w.shape)))
    e[2].record(stream)
    torch.cuda.synchronize()
    fwd = e[0].elapsed_time(e[1])
    rev = e[1].elapsed_time(e[2])
    sol.close()
    return {"metric": "coupled adjoint: reverse-pass wall time per step", "value": rev / steps,
            "unit": "ms/step", "higher_is_better": False,
            "config": {"workload": f"rough ellipsoid {n}^3, per-voxel log E, log g_c, "
                                   f"log D ~ N(0, 0.1^2), FP64, checkpoint every 5 steps, "
                                   f"loss with random seeds on the final (c, F, d)",
                       "steps": steps, "warmup": warmup},
            "forward_ms_per_step": fwd / steps, "reverse_over_forward": rev / fwd,
            "adjoint_stats": st, "grad_max": {k: float(v.abs().max()) for k, v in g.items()}}


def batch_mode(count, steps, warmup):
    """Many independent particle RVEs of uneven size: one batched coupled step (members
    on their own streams, driven concurrently) against the same members stepped one by
    one.  Returns aggregate voxel-steps/s of both."""
    import torch
    from paper_2411_16583_gb300 import binding as B, synth as S
    ws = S.sphere_batch(count=count, nsteps=20, seed=0)
    V = sum(w.nvox for w in ws)
    mk = lambda: [B.from_workload(w, precision=B.FG_MIXED) for w in ws]
    seq = mk()
    for s_, w in zip(seq, ws):
        s_.autotune()
    for _ in range(warmup):
        for s_, w in zip(seq, ws):
            s_.step(w.dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        for s_, w in zip(seq, ws):
            s_.step(w.dt)
    torch.cuda.synchronize()
    t_seq = (time.perf_counter() - t0) / steps
    for s_ in seq:
        s_.close()
    mem = mk()
    for s_ in mem:
        s_.autotune()
    batch = B.Batch(mem)
    for _ in range(warmup):
        batch.step(1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        st = batch.step(1.0)
    torch.cuda.synchronize()
    t_b = (time.perf_counter() - t0) / steps
    # the members' FP32 mechanical operator at their current states: grouped launches (one
    # per pass over every member of a grid, from a device table of pass arguments) against
    # the members' own launches
    ms, info = batch.time_apply(prec=1, n=20)
    batch.close()
    for s_ in mem:
        s_.close()
    names = ("grouped_graph", "grouped", "members_one_stream", "members_own_streams")
    apply = {"kind": "FP32 mechanical operator application of all members (Eq. mechanicalsolve)",
             "applications": 20, "groups": info[0], "launches_grouped": info[1],
             "launches_members": info[2],
             "ms": dict(zip(names, ms)),
             "voxel_applies_per_s": {k: V / (t * 1e-3) for k, t in zip(names, ms)}}
    apply["grouped_graph_over_own_streams"] = ms[3] / ms[0]
    return {"mode": "batch", "rves": len(ws), "voxels": V, "steps": steps, "warmup": warmup,
            "apply": apply,
            "sizes": sorted({w.shape[0] for w in ws}),
            "batched_voxel_steps_per_s": V / t_b, "sequential_voxel_steps_per_s": V / t_seq,
            "batched_ms_per_step": t_b * 1e3, "sequential_ms_per_step": t_seq * 1e3,
            "speedup": t_seq / t_b, "cg_mech_total": sum(x["cg_mech"] for x in st),
            "cg_graph_replays": sum(x["cg_graph_replays"] for x in st)}


def reference_arm(a, rank, world):
    """The CPU oracle as it stands, on this arm's workload, metric and unit."""
    if rank != 0:
        return
    w = _workload(a.n, seed=0)
    budget = max(3.0, min(a.cpu_seconds, 30.0))
    # one sample of every operator first (the mechanical one, about 19 s at 256^3, is not
    # timed again); each warm-up and timed step then times the projection and the
    # chemistry operator afresh, so the run ends within a few minutes
    _, _, first = oracle_step_seconds(w, budget, DEFAULT_STEP_PROFILE)
    reuse = {"mech": first["mech"]}
    total, desc = 0.0, None
    for k in range(a.warmup + a.steps):
        s, desc, _ = oracle_step_seconds(w, 0.0, DEFAULT_STEP_PROFILE, reuse=reuse)
        if k >= a.warmup:
            total += s
    per_step = total / a.steps
    value = w.nvox / per_step
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(a),
                   "precision": "FP64 (the CPU oracle); per-operator times on the full fields "
                                "times the FP64 form's operator counts of the window's first "
                                "step",
                   "voxels": w.nvox},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
