"""Benchmark: coupled time steps of the FFT chemo-mechanical fracture method on GB300.

Default workload: the 256^3 rough ellipsoidal particle (semi-axes 100/80/70 voxels,
roughness std 3 / correlation 8, influx band 8 voxels, Gaussian concentration perturbation
std 0.02), mixed FP32/FP64 precision, Newton tolerance 1e-9.  One bench step = one coupled
time step (Alg. 4: chemistry Newton-CG, then staggered mechanics Newton-CG and phase-field
PCG) through the C ABI.  Inputs are resident on the device before the timed region; the
working set (~15 GB) is far larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead.
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


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=256, help="grid edge of the particle workload")
    p.add_argument("--fp64-steps", type=int, default=1, help="FP64 comparison steps (0: skip)")
    p.add_argument("--cpu-seconds", type=float, default=20.0, help="oracle sample budget")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def _workload(n, seed):
    from paper_2411_16583_gb300 import synth as S
    if n == 256:
        return S.ellipsoid256(seed=seed)
    f = n / 256.0
    return S.ellipsoid(n=n, axes=(100 * f, 80 * f, 70 * f), rough_std=3 * f, rough_corr=8 * f,
                       band=max(1, round(8 * f)), nsteps=100, seed=seed, c_perturb=0.02)


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
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_baseline(w, budget_s):
    """The oracle as it stands on a bounded sample of the same workload: repeated FP64
    mechanical operator applications on the full 256^3 fields (the operator a coupled step
    spends its time in), single process."""
    import numpy as np
    from oracle import fg_oracle as O
    from paper_2411_16583_gb300 import synth as S
    prm = O.make_params([O.Phase(**vars(p)) for p in w.phases], w.phase_id, w.h, gc=w.gc,
                        lc=w.lc, RT=w.RT, cmax=w.cmax)
    F, c, d = S.random_state(w.shape, seed=1, f_amp=0.01, c_lo=0.01, c_hi=0.3, d_hi=0.0)
    x = S.random_tensor_field(w.shape, 2).reshape((3, 3) + w.shape)
    n, t0 = 0, time.perf_counter()
    while True:
        O.mech_apply(F, c, d, prm, x)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = (time.perf_counter() - t0) / n
    return {"voxel_applies_per_s": w.nvox / dt, "seconds_per_apply": dt, "applies": n,
            "cores": int(os.environ.get("OMP_NUM_THREADS", "0") or 0) or 1}


def main():
    a = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return reference_arm(a, rank, world)
    import numpy as np
    import torch
    from paper_2411_16583_gb300 import binding as B
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = _workload(a.n, seed=rank)
    stream = torch.cuda.current_stream()
    sol = B.from_workload(w, precision=B.FG_MIXED, stream=stream.cuda_stream)
    V = w.nvox
    for _ in range(a.warmup):
        sol.step(w.dt)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    stats = []
    with Clocks(local) as clk:
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            stats.append(sol.step(w.dt))
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1) / a.steps
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # fused matvec rates (FP32 in the mixed context)
    mech32_ms = sol.time_apply(B.OP_MECH, 1, 20)
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
    line = {
        "metric": METRIC,
        "value": V * world / (ms * 1e-3),
        "unit": "voxel-steps/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 inner / f64 outer",
        "data": "synthetic",
        "config": {"workload": f"rough ellipsoid particle {a.n}^3, mixed FP32/FP64, Newton tol 1e-9",
                   "voxels": V, "l2": "working set >> L2 (no flush needed)"},
        "matvec": {"mech_fp32_voxel_applies_per_s": V / (mech32_ms * 1e-3),
                   "mech_fp32_ms": mech32_ms},
        "step_stats": stats[-1],
        "clocks": clk.summary(),
        "peaks_source": src,
    }
    line.update(out)
    if not a.no_cpu_baseline:
        cb = cpu_baseline(w, a.cpu_seconds)
        line["cpu_baseline"] = {"value": cb["voxel_applies_per_s"], "unit": "voxel-applies/s",
                                "cores": cb["cores"], "kind": "oracle",
                                "sample": f"{cb['applies']} FP64 mechanical operator applications "
                                          f"at {a.n}^3 (numpy oracle)"}
    print(json.dumps(line))


def reference_arm(a, rank, world):
    if rank != 0:
        return
    print(json.dumps({"impl": "reference", "unavailable": "not implemented yet"}))


if __name__ == "__main__":
    main()
