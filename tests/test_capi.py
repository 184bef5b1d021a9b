"""The C-ABI library loads and exports every entry point ``include/fg.h`` declares, and
its host-side argument checks return the documented error codes (through the host
emulation build, so no GPU is needed)."""
import os
import re

import numpy as np
import pytest

from paper_2411_16583_gb300 import binding as B, build, synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fg_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert set(declared_symbols()) == set(B.EXPORTS)


@pytest.mark.parametrize("which", ["gpu", "emu"])
def test_library_exports_every_declared_symbol(which):
    path = build.build_gpu() if which == "gpu" else build.build_emu()
    import ctypes
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


@pytest.fixture(scope="module")
def emu():
    return B.load_library(build.build_emu())


def _disc(n=16):
    return S.disc2d(n=n, radius=6.0, band=3, nsteps=10)


def test_invalid_arguments(emu):
    w = _disc()
    with pytest.raises(B.FgError) as e:  # odd nx
        B.Solver((1, 16, 15), w.h, w.phases, np.zeros((1, 16, 15)), np.zeros((1, 16, 15)), lib=emu)
    assert e.value.code == -1
    with pytest.raises(B.FgError) as e:  # a length that is not compiled in
        B.Solver((1, 16, 18), w.h, w.phases, np.zeros((1, 16, 18)), np.zeros((1, 16, 18)), lib=emu)
    assert e.value.code == -1
    bad = w.phase_id.copy()
    bad[0, 0, 0] = 7  # phase id out of range
    with pytest.raises(B.FgError) as e:
        B.Solver(w.shape, w.h, w.phases, bad, w.cdot_B, lib=emu)
    assert e.value.code == -1
    mixed_laws = S.default_phases()
    mixed_laws[1].law = S.LAW_SVK
    with pytest.raises(B.FgError) as e:  # one law per context
        B.Solver(w.shape, w.h, mixed_laws, w.phase_id, w.cdot_B, lib=emu)
    assert e.value.code == -1
    with pytest.raises(B.FgError) as e:  # initial concentration outside (0, 1)
        B.Solver(w.shape, w.h, w.phases, w.phase_id, w.cdot_B, c_init=np.full(w.shape, 1.2), lib=emu)
    assert e.value.code == -5
    s_ = B.from_workload(w, lib=emu)
    try:  # F and Fbar of fg_displacement come together
        u = np.empty((3,) + w.shape)
        F = np.zeros((9,) + w.shape)
        for call in (lambda: emu.fg_displacement(s_.ctx, B._ptr(F), None, B._ptr(u), 0),
                     lambda: emu.fg_displacement(s_.ctx, None, B._ptr(np.eye(3)), B._ptr(u), 0)):
            with pytest.raises(B.FgError, match="fg_displacement"):
                s_._check(call())
    finally:
        s_.close()
    bad_smax = np.zeros(w.shape)
    bad_smax.flat[3] = np.inf  # sigma_max(x) = sigma_max exp(log_smax) must stay finite
    with pytest.raises(B.FgError, match="sigma_max") as e:
        B.Solver(w.shape, w.h, w.phases, w.phase_id, w.cdot_B, log_smax=bad_smax, lib=emu)
    assert e.value.code == -1
    with pytest.raises(B.FgError, match="cg_indefinite") as e:  # modes 0, 1, 2 only
        B.from_workload(w, lib=emu, cg_indefinite=3)
    assert e.value.code == -1
    with pytest.raises(B.FgError, match="no recorded steps") as e:  # adjoint without a tape
        s_ = B.from_workload(w, lib=emu)
        try:
            s_.adjoint()
        finally:
            s_.close()
    with pytest.raises(B.FgError, match="fg_tape_begin") as e:
        s_ = B.from_workload(w, lib=emu)
        try:
            s_.tape(0)
        finally:
            s_.close()
    s_ = B.from_workload(w, lib=emu)
    try:
        with pytest.raises(B.FgError, match="fg_set_stress_control"):
            s_._check(emu.fg_set_stress_control(s_.ctx, 512, None))
        s_.stress_control(np.eye(3, dtype=bool), np.zeros((3, 3)))
        s_.step(w.dt)
        s_.tape(1)
        s_.step(w.dt)
        _, _, st = s_.adjoint()  # the adjoint covers mixed control too
        assert st["steps"] == 1
    finally:
        s_.close()
    assert emu.fg_supported_size(64) == 1 and emu.fg_supported_size(18) == 0


def test_iteration_cap_reports_noconv_and_keeps_state(emu):
    w = _disc()
    sol = B.from_workload(w, lib=emu, max_cg=2)
    c0 = sol.get(B.FIELD_C)
    st = sol.step(w.dt, check=False)
    assert st["status"] == -4
    np.testing.assert_array_equal(sol.get(B.FIELD_C), c0)  # state left at the step start
    sol.close()


def test_nan_input_is_reported(emu):
    w = _disc()
    sol = B.from_workload(w, lib=emu)
    F = sol.get(B.FIELD_F)
    F[0, 0, 0, 3, 3] = np.nan
    sol.set(B.FIELD_F, F)
    st = sol.step(w.dt, check=False)
    assert st["status"] in (-5, -6)
    sol.close()


def test_save_load_restarts_bit_identically(emu, tmp_path):
    """A context restored from a restart file after one step takes the second step exactly
    as the context that wrote it; a file for another grid is refused."""
    w = S.disc2d(n=16, radius=6.0, band=3, nsteps=10)
    a = B.from_workload(w, lib=emu)
    a.step(w.dt)
    path = str(tmp_path / "state.fg")
    a.save(path)
    b = B.from_workload(w, lib=emu)
    b.load(path)
    a.step(w.dt)
    b.step(w.dt)
    for f in (B.FIELD_C, B.FIELD_F, B.FIELD_D, B.FIELD_H):
        np.testing.assert_array_equal(a.get(f), b.get(f))
    np.testing.assert_array_equal(np.array(a.residual()), np.array(b.residual()))
    w2 = S.disc2d(n=24, radius=6.0, band=3, nsteps=10)
    c = B.from_workload(w2, lib=emu)
    with pytest.raises(B.FgError, match="grid"):
        c.load(path)
    with pytest.raises(B.FgError, match="cannot open"):
        c.load(str(tmp_path / "missing.fg"))
    for s_ in (a, b, c):
        s_.close()


def test_state_writes_are_refused_while_the_tape_holds_steps(emu, tmp_path):
    """fg_adjoint recomputes the recorded trajectory from its checkpoints, so fg_set_field
    and fg_load, which would make the stored state jump between two recorded steps, are
    refused while the tape holds steps; a new tape (fg_tape_begin) allows them again."""
    w = _disc()
    s_ = B.from_workload(w, lib=emu)
    try:
        s_.step(w.dt)
        path = str(tmp_path / "state.fg")
        s_.save(path)
        s_.tape(1)
        s_.step(w.dt)
        c = s_.get(B.FIELD_C)
        with pytest.raises(B.FgError, match="fg_set_field: steps are recorded") as e:
            s_.set(B.FIELD_C, c * 0.5)
        assert e.value.code == -1
        with pytest.raises(B.FgError, match="fg_load: steps are recorded") as e:
            s_.load(path)
        assert e.value.code == -1
        np.testing.assert_array_equal(s_.get(B.FIELD_C), c)  # nothing was written
        s_.adjoint()
        s_.tape(1)  # an empty tape
        s_.load(path)
        s_.set(B.FIELD_C, c)
    finally:
        s_.close()


def test_save_load_keeps_mixed_stress_control(emu, tmp_path):
    """The restart file carries the stress-control mask and the prescribed mean stress, so a
    context restored after a mixed-control step steps on as the one that wrote it."""
    w = _disc()
    mask = np.zeros((3, 3), dtype=bool)
    mask[1, 1] = True
    Pbar = np.zeros((3, 3))
    a = B.from_workload(w, lib=emu)
    a.stress_control(mask, Pbar)
    a.step(w.dt)
    path = str(tmp_path / "mixed.fg")
    a.save(path)
    b = B.from_workload(w, lib=emu)  # full strain control until the file is read
    b.load(path)
    a.step(w.dt)
    b.step(w.dt)
    for f in (B.FIELD_C, B.FIELD_F, B.FIELD_D, B.FIELD_H):
        np.testing.assert_array_equal(a.get(f), b.get(f))
    c = B.from_workload(w, lib=emu)
    c.step(w.dt)
    c.step(w.dt)
    assert np.abs(c.get(B.FIELD_F) - a.get(B.FIELD_F)).max() > 1e-9  # the mask matters
    for s_ in (a, b, c):
        s_.close()


@pytest.mark.parametrize("mode,offset,faults", [
    ("end", 0, False), ("end", 63, False), ("end", 64, True),
    ("start", 0, False), ("start", 63, False), ("start", -1, True)])
def test_emulated_memory_guards_fault_out_of_bounds(mode, offset, faults):
    """The host emulation places every emulated device buffer against an inaccessible page,
    so the emulated kernels of the other tests run bounds-checked: a write one byte past
    the end (or, with FG_EMU_GUARD=start, one byte before the start) of a buffer faults.
    Checked in a child process on the CPU."""
    import signal
    import subprocess
    import sys
    path = build.build_emu()
    code = ("import ctypes, sys; lib = ctypes.CDLL(sys.argv[1]); "
            "lib.fg_emu_guard_probe.argtypes = [ctypes.c_longlong]; "
            "sys.exit(lib.fg_emu_guard_probe(int(sys.argv[2])))")
    env = dict(os.environ, FG_EMU_GUARD=mode)
    r = subprocess.run([sys.executable, "-c", code, path, str(offset)], env=env,
                       capture_output=True, timeout=120)
    assert r.returncode == (-signal.SIGSEGV if faults else 0), r.stderr.decode()[-500:]


def test_emulated_kernels_in_bounds_below_start():
    """The emulated operators, coupled steps, batch and mechanical adjoint rerun with every
    buffer starting on its guard page (FG_EMU_GUARD=start): no kernel indexes below zero.
    (The default placement, guard after the end, covers the whole emulated suite.)"""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, FG_EMU_GUARD="start")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_emu_kernels.py", "-q",
                        "-p", "no:cacheprovider", "-k",
                        "operators or coupled_step_matches or batch or homogeneous or mech_adjoint"],
                       cwd=root, env=env, capture_output=True, timeout=900)
    assert r.returncode == 0, r.stdout.decode()[-2000:]


@pytest.mark.parametrize("prec", [B.FG_FP64, B.FG_MIXED])
def test_inverting_load_reports_domain_and_keeps_state(emu, prec):
    """A macroscopic load with det F-bar < 0 puts every voxel outside the domain of the
    law: the step returns FG_ERR_DOMAIN, the stored state (F, c, d, H) is exactly the one
    before the step, and the next valid step runs."""
    w = S.disc2d()
    sol = B.from_workload(w, lib=emu, precision=prec)
    sol.step(w.dt)
    fields = (B.FIELD_F, B.FIELD_C, B.FIELD_D, B.FIELD_H)
    before = [sol.get(f).copy() for f in fields]
    with pytest.raises(B.FgError) as e:
        sol.step(w.dt, np.diag([-1.0, 1.0, 1.0]))
    assert e.value.code == -5
    for f, b in zip(fields, before):
        np.testing.assert_array_equal(sol.get(f), b)
    assert sol.step(w.dt)["status"] == 0
    sol.close()
