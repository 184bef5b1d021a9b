"""fg_mech_apply_noalloc: the operator application for callers that cannot allocate GPU
memory (their device memory belongs to a host framework's pool or a fixed budget).  It
keeps all scratch in one static device array.  Checked against fg_apply (FG_OP_MECH,
FP32) and against the CPU oracle's operator on two calls in a row with different inputs,
and for its size limit.  This file is
collected last so that a run stopping at the first failure has run every other test."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fg_oracle as O
from paper_2411_16583_gb300 import binding as B, synth as S
from tests.helpers import TOL_APPLY_FP32, oracle_params, rel_err

pytestmark = pytest.mark.gpu

SHAPE = (16, 32, 64)
H = (1.0e-7, 1.1e-7, 0.9e-7)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_apply_matches_fg_apply_twice():
    assert torch.cuda.is_available()
    lib = B.load_library()
    pid = S.random_phase_map(SHAPE, 1)
    phases = S.default_phases()
    phases[1].E = 2e9
    sol = B.Solver(SHAPE, H, phases, pid, np.zeros(SHAPE), lib=lib, precision=B.FG_MIXED)
    F, c, d = S.random_state(SHAPE, seed=4)
    for f, v in ((B.FIELD_F, F), (B.FIELD_C, c), (B.FIELD_D, d)):
        sol.set(f, v)
    prm = oracle_params(phases, pid, H)
    E = np.array([p.E for p in phases])[pid]
    nu = np.array([p.nu for p in phases])[pid]
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    Om = np.array([p.Omega for p in phases])[pid]
    c0 = np.array([p.c0 for p in phases])[pid]
    dev = {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()
           for k, v in dict(F=F, c=c, d=d, lam=lam, mu=mu, Om=Om, c0=c0).items()}
    for seed in (7, 8):  # two calls in a row share the static scratch
        x = torch.from_numpy(S.random_tensor_field(SHAPE, seed)).to("cuda", torch.float32)
        y_ref = torch.empty_like(x)
        dot_ref = sol.apply(B.OP_MECH, x, y_ref, 1)
        y = torch.full_like(x, float("nan"))
        dot = C.c_double()
        torch.cuda.synchronize()
        rc = lib.fg_mech_apply_noalloc(SHAPE[2], SHAPE[1], SHAPE[0], *H, _ptr(dev["F"]),
                                       _ptr(dev["c"]), _ptr(dev["d"]), _ptr(dev["lam"]),
                                       _ptr(dev["mu"]), _ptr(dev["Om"]), _ptr(dev["c0"]),
                                       _ptr(x), _ptr(y), C.byref(dot), None)
        assert rc == 0, lib.fg_last_error()
        assert rel_err(y.cpu().numpy(), y_ref.cpu().numpy()) < TOL_APPLY_FP32
        assert abs(dot.value - dot_ref) <= TOL_APPLY_FP32 * abs(dot_ref)
        Fo = F.reshape((3, 3) + SHAPE)
        ref = O.mech_apply(Fo, c, d, prm, x.double().cpu().numpy().reshape(Fo.shape))
        assert rel_err(y.cpu().numpy().reshape(ref.shape), ref) < TOL_APPLY_FP32
    sol.close()


def test_noalloc_apply_rejects_grids_beyond_its_static_size():
    lib = B.load_library()
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    zf = torch.zeros(1, dtype=torch.float32, device="cuda")
    p = [_ptr(z)] * 7
    rc = lib.fg_mech_apply_noalloc(128, 64, 64, *H, *p, _ptr(zf), _ptr(zf), None, None)
    assert rc == -1 and b"64" in lib.fg_last_error()
