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


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=256, help="grid edge of the particle workload")
    p.add_argument("--nz", type=int, default=0, help="override the z extent (profiling cases)")
    p.add_argument("--fp64-steps", type=int, default=1, help="FP64 comparison steps (0: skip)")
    p.add_argument("--cpu-seconds", type=float, default=20.0, help="oracle sample budget")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--adjoint", action="store_true",
                   help="time the coupled adjoint (128^3 ellipsoid with log fields, FP64, "
                        "checkpoints every 5 steps) instead of the step benchmark")
    p.add_argument("--batch", type=int, default=0,
                   help="batched RVEs: N particles of seeded sizes {48,64,80,96}^3 (0: off)")
    return p.parse_args()


def _workload(n, seed, nz=0):
    from paper_2411_16583_gb300 import synth as S
    if n == 256 and not nz:
        return S.ellipsoid256(seed=seed)
    f = n / 256.0
    shape = (nz, n, n) if nz else None
    axes = (100 * f, 80 * f, min(70 * f, 0.4 * nz) if nz else 70 * f)
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
# the first coupled step of this workload on the FP64 path, whose Krylov iterations follow
# the oracle's (measured on a GB300 with the buffer at 1e-2 of the particle's stiffness).
DEFAULT_STEP_PROFILE = {"cg_mech": 549, "newton_mech": 3, "stag": 1, "cg_chem": 746,
                        "newton_chem": 8, "cg_pff": 0}


def oracle_step_seconds(w, budget_s, profile):
    """Times the oracle's operators on the full-size fields of workload w (a bounded
    sample, about budget_s seconds) and combines them with the operator counts of one
    coupled step.  Returns (seconds per step, description of the sample)."""
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
    times, counts = {}, {}
    t_start = time.perf_counter()
    share = budget_s / len(ops)
    for k, f in ops.items():
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
    return step, desc


def _cores():
    try:
        import numpy as np  # noqa: F401
        return int(os.environ.get("OMP_NUM_THREADS") or 1)
    except Exception:
        return 1


def cufft_comparator(sol, w, reps=10, device="cuda"):
    """The FP32 Neo-Hookean mechanical operator y = G : F^-1[F[K : x]] of the stored state
    assembled from torch element-wise kernels and torch.fft (cuFFT), unfused: the timed
    comparator for the fused apply.  Returns (ms per apply, max |y - y_fused| / max |y|)."""
    import numpy as np
    import torch
    from paper_2411_16583_gb300 import binding as B
    dev = torch.device(device)
    nz, ny, nx = w.shape
    V = w.nvox
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev, torch.float32)
    F = f32(sol.get(B.FIELD_F).reshape(3, 3, V))
    c = f32(sol.get(B.FIELD_C).ravel())
    d = f32(sol.get(B.FIELD_D).ravel())
    pid = w.phase_id.ravel()
    tab = lambda attr: f32(np.array([getattr(p, attr) for p in w.phases])[pid])
    E, nu, Om, c0 = tab("E"), tab("nu"), tab("Omega"), tab("c0")
    if w.log_E is not None:
        E = E * f32(np.exp(w.log_E.ravel()))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    a = (1 + Om * (c - c0)) ** (-1.0 / 3.0)
    g = (1 - d) ** 2
    Fe = (a * F).permute(2, 0, 1)                       # (V, 3, 3)
    # F_e^-T = cof(F_e) / det F_e, written out (element-wise kernels only)
    f = [[Fe[:, i, j] for j in range(3)] for i in range(3)]
    cof = torch.stack([torch.stack([f[(i + 1) % 3][(j + 1) % 3] * f[(i + 2) % 3][(j + 2) % 3]
                                    - f[(i + 1) % 3][(j + 2) % 3] * f[(i + 2) % 3][(j + 1) % 3]
                                    for j in range(3)], dim=1) for i in range(3)], dim=1)
    J = (Fe[:, 0, :] * cof[:, 0, :]).sum(dim=1)
    Bt = cof / J[:, None, None]
    lnJ = torch.log(J)
    s1, s2, s3 = (g * a * a)[:, None, None], (mu - lam * lnJ)[:, None, None], lam[:, None, None]

    def tangent(X):                                     # X (V, 3, 3): K : X
        M = Bt @ X.transpose(1, 2) @ Bt
        tr = (Bt * X).sum(dim=(1, 2))[:, None, None]
        return s1 * (mu[:, None, None] * X + s2 * M + s3 * tr * Bt)

    def freq(n, h):
        k = torch.arange(n, device=dev, dtype=torch.float64)
        q = 2 * np.pi * k / n
        return (2.0 / h) * torch.sin(q / 2), torch.cos(q / 2)
    (sx, cx), (sy, cy), (sz, cz) = freq(nx, w.h[0]), freq(ny, w.h[1]), freq(nz, w.h[2])
    sx, cx = sx[: nx // 2 + 1], cx[: nx // 2 + 1]
    cx[-1] = 0.0 if nx % 2 == 0 else cx[-1]
    cy[ny // 2] = 0.0 if ny % 2 == 0 else cy[ny // 2]
    cz[nz // 2] = 0.0 if nz % 2 == 0 else cz[nz // 2]
    Z, Y, X_ = torch.meshgrid(torch.arange(nz, device=dev), torch.arange(ny, device=dev),
                              torch.arange(nx // 2 + 1, device=dev), indexing="ij")
    n = torch.stack([sx[X_] * cy[Y] * cz[Z], cx[X_] * sy[Y] * cz[Z], cx[X_] * cy[Y] * sz[Z]]).float()
    n2 = (n * n).sum(0)
    inv = torch.where(n2 > 0, 1.0 / n2, torch.zeros_like(n2))

    def apply(x):                                       # x (9, V)
        tau = tangent(x.reshape(3, 3, V).permute(2, 0, 1)).permute(1, 2, 0).reshape(3, 3, nz, ny, nx)
        T = torch.fft.rfftn(tau, dim=(-3, -2, -1))
        An = torch.einsum("imzyx,mzyx->izyx", T, n.to(T.dtype))
        Y_ = torch.einsum("izyx,jzyx->ijzyx", An * inv, n.to(T.dtype))
        return torch.fft.irfftn(Y_, s=(nz, ny, nx), dim=(-3, -2, -1)).reshape(9, V)
    x = torch.randn(9, V, dtype=torch.float32, generator=torch.Generator().manual_seed(0)).to(dev)
    yf = torch.empty_like(x)
    sol.apply(B.OP_MECH, x, yf, prec=1)
    y = apply(x)
    diff = float((y - yf).abs().max() / yf.abs().max())
    if dev.type != "cuda":
        return None, diff
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream()
    e0.record(cur)
    for _ in range(reps):
        y = apply(x)
    e1.record(cur)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, diff


def main():
    a = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return reference_arm(a, rank, world)
    if a.batch:
        return batch_mode(a)
    if a.adjoint:
        return adjoint_mode(a)
    import numpy as np
    import torch
    from paper_2411_16583_gb300 import binding as B
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = _workload(a.n, seed=rank, nz=a.nz)
    stream = torch.cuda.current_stream()
    sol = B.from_workload(w, precision=B.FG_MIXED, stream=stream.cuda_stream)
    V = w.nvox
    tuned_ms = sol.autotune()
    for _ in range(a.warmup):
        sol.step(w.dt)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for s in range(5):
        sol.profile(s, True)
    stats = []
    with Clocks(local) as clk:
        barrier()
        l0 = B.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            stats.append(sol.step(w.dt))
        e1.record(stream)
        barrier()
        launches = B.kernel_launches() - l0
    ms = e0.elapsed_time(e1) / a.steps
    prof = {s: sol.profile_read(s) for s in range(5)}
    for s in range(5):
        sol.profile(s, False)
    ms = max_over_ranks(ms, dist, "cuda")

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

    # fused matvec rates: FP32 operator of the mixed context, and the unfused cuFFT
    # comparator of the same operator
    mech32_ms = sol.time_apply(B.OP_MECH, 1, 20)
    comparator = None
    if w.phases[0].law == B.FG_NEOHOOKE and rank == 0:
        try:
            cms, cdiff = cufft_comparator(sol, w)
            comparator = {"kind": "torch element-wise + torch.fft (cuFFT), unfused, FP32",
                          "ms_per_apply": cms, "voxel_applies_per_s": V / (cms * 1e-3),
                          "max_rel_diff_vs_fused": cdiff}
        except torch.cuda.OutOfMemoryError as e:  # noqa: F841
            comparator = {"unavailable": "out of device memory"}
    sol.close()
    out = {}
    if a.fp64_steps > 0 and rank == 0:
        sol64 = B.from_workload(w, precision=B.FG_FP64, stream=stream.cuda_stream)
        mech64_ms = sol64.time_apply(B.OP_MECH, 0, 5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s64 = [sol64.step(w.dt) for _ in range(a.fp64_steps)]
        torch.cuda.synchronize()
        out["fp64_step_ms"] = (time.perf_counter() - t0) * 1e3 / a.fp64_steps
        out["fp64_step_stats"] = s64[-1]
        out["mech_fp64_voxel_applies_per_s"] = V / (mech64_ms * 1e-3)
        sol64.close()
    if rank != 0:
        return
    peaks, src = _peaks()
    sb = site_bytes(w.shape[2])
    sites = {}
    for s, (n, t, vol) in prof.items():
        if n:
            sites[SITE_NAMES[s]] = {"launches": n, "total_ms": t, "volumes": vol,
                                    "us_per_volume": t * 1e3 / vol,
                                    "alg_bytes_per_voxel": sb[s],
                                    "gbs": sb[s] * V * vol / (t * 1e-3) / 1e9}
    dom = max((s for s in prof if prof[s][0]), key=lambda s: prof[s][1])
    n_dom, t_dom, vol_dom = prof[dom]
    avg_dom = t_dom / n_dom * 1e-3           # seconds per launch
    ach = sb[dom] * V * vol_dom / (t_dom * 1e-3) / 1e9
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
        "config": {"workload": f"rough ellipsoid particle {a.n}^3 (coupled step, mixed "
                               f"FP32 Krylov / FP64 Newton, tol 1e-9)",
                   "voxels": V, "l2": "inputs larger than L2 (no flush)"},
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": SITE_NAMES[dom], "achieved": ach,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                     "peak_source": src,
                     "alg_bytes_per_launch": sb[dom] * V * vol_dom / n_dom,
                     "avg_launch_us": avg_dom * 1e6,
                     "traffic": _traffic(dom, w.shape[2], V * vol_dom / n_dom)},
        "kernels": sites,
        "matvec": {"mech_fp32_voxel_applies_per_s": V / (mech32_ms * 1e-3),
                   "mech_fp32_ms": mech32_ms, "cufft_comparator": comparator},
        "step_stats": stats[-1],
        "autotuned_apply_ms": tuned_ms,
        "clocks": clk.summary(),
    }
    line.update(out)
    if not a.no_cpu_baseline:
        # the oracle is an FP64 method: its step takes the FP64 form's operator counts (of
        # this run when it timed an FP64 step, else those recorded at 256^3)
        counts = out.get("fp64_step_stats") or DEFAULT_STEP_PROFILE
        prof_counts = {k: counts[k] for k in DEFAULT_STEP_PROFILE}
        secs, desc = oracle_step_seconds(w, a.cpu_seconds, prof_counts)
        line["cpu_baseline"] = {"value": V / secs, "unit": UNIT, "cores": _cores(),
                                "kind": "oracle", "sample": desc}
    print(json.dumps(line))


def adjoint_mode(a):
    """Forward steps with a tape, then the reverse pass for dL/dlog(E, g_c, D) of a loss
    with random seeds on the final state; both timed with CUDA events on the context's
    stream (FP64 throughout)."""
    import torch
    from paper_2411_16583_gb300 import binding as B, synth as S
    n = a.n if a.n != 256 else 128
    w = S.with_log_fields(S.ellipsoid(n=n, axes=(50 * n / 128, 40 * n / 128, 35 * n / 128),
                                      rough_std=1.5 * n / 128, rough_corr=4 * n / 128,
                                      band=max(1, round(8 * n / 128)), nsteps=50,
                                      phases=S.default_phases(buffer_E=S.BENCH_BUFFER_E)),
                          std=0.1)
    stream = torch.cuda.current_stream()
    sol = B.from_workload(w, precision=B.FG_FP64, stream=stream.cuda_stream)
    for _ in range(a.warmup):
        sol.step(w.dt)
    sol.tape(5)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record(stream)
    for _ in range(a.steps):
        sol.step(w.dt)
    e[1].record(stream)
    # a loss with seeded random dL/d(c, F, d) on the final state: every adjoint solve
    # runs (the fracture energy is zero until damage starts)
    import numpy as np
    rng = np.random.default_rng(0)
    val, g, st = sol.adjoint(B.FG_LOSS_SEEDS, seed_c=rng.standard_normal(w.shape),
                             seed_F=rng.standard_normal((3, 3) + w.shape),
                             seed_d=rng.standard_normal(w.shape))
    e[2].record(stream)
    torch.cuda.synchronize()
    fwd = e[0].elapsed_time(e[1])
    rev = e[1].elapsed_time(e[2])
    print(json.dumps({"metric": "coupled adjoint: reverse-pass wall time per step", "value":
                      rev / a.steps, "unit": "ms/step", "higher_is_better": False,
                      "config": {"workload": f"rough ellipsoid {n}^3, per-voxel log E, log g_c, "
                                 f"log D ~ N(0, 0.1^2), FP64, checkpoint every 5 steps, "
                                 f"loss with random seeds on the final (c, F, d)",
                                 "steps": a.steps, "warmup": a.warmup},
                      "forward_ms_per_step": fwd / a.steps, "loss": val, "adjoint_stats": st,
                      "grad_max": {k: float(abs(v).max()) for k, v in g.items()}}))
    sol.close()


def batch_mode(a):
    """Many independent particle RVEs of uneven size: one batched coupled step (members
    on their own streams, driven concurrently) against the same members stepped one by
    one.  Reports aggregate voxel-steps/s of both."""
    import torch
    from paper_2411_16583_gb300 import binding as B, synth as S
    ws = S.sphere_batch(count=a.batch, nsteps=20, seed=0)
    V = sum(w.nvox for w in ws)
    mk = lambda: [B.from_workload(w, precision=B.FG_MIXED) for w in ws]
    seq = mk()
    for s_, w in zip(seq, ws):
        s_.autotune()
    for _ in range(a.warmup):
        for s_, w in zip(seq, ws):
            s_.step(w.dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        for s_, w in zip(seq, ws):
            s_.step(w.dt)
    torch.cuda.synchronize()
    t_seq = (time.perf_counter() - t0) / a.steps
    for s_ in seq:
        s_.close()
    mem = mk()
    for s_ in mem:
        s_.autotune()
    batch = B.Batch(mem)
    for _ in range(a.warmup):
        batch.step(1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        st = batch.step(1.0)
    torch.cuda.synchronize()
    t_b = (time.perf_counter() - t0) / a.steps
    batch.close()
    print(json.dumps({"mode": "batch", "rves": len(ws), "voxels": V,
                      "sizes": sorted({w.shape[0] for w in ws}),
                      "batched_voxel_steps_per_s": V / t_b, "sequential_voxel_steps_per_s": V / t_seq,
                      "batched_ms_per_step": t_b * 1e3, "sequential_ms_per_step": t_seq * 1e3,
                      "speedup": t_seq / t_b, "cg_mech_total": sum(x["cg_mech"] for x in st)}))


def reference_arm(a, rank, world):
    """The CPU oracle as it stands, on this arm's workload, metric and unit."""
    if rank != 0:
        return
    w = _workload(a.n, seed=0)
    budget = max(3.0, min(a.cpu_seconds, 30.0))
    secs, desc = None, None
    total = 0.0
    for _ in range(a.warmup + a.steps):
        s, desc = oracle_step_seconds(w, budget / 3, DEFAULT_STEP_PROFILE)
        total += s
        secs = s
    per_step = total / (a.warmup + a.steps)
    value = w.nvox / per_step
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"rough ellipsoid particle {a.n}^3 (coupled step, oracle FP64)",
                   "voxels": w.nvox},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
