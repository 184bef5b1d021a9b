"""Thin ctypes binding of the C ABI in ``include/fg.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``_lib/libfg.so``; this module only
converts arguments.  Loading fails loudly when the library has not been built: there is
no Python or CPU fallback.  PyTorch is used for device memory and the current stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libfg.so")

FG_OK = 0
ERRORS = {-1: "FG_ERR_INVALID", -2: "FG_ERR_OOM", -3: "FG_ERR_CUDA", -4: "FG_ERR_NOCONV",
          -5: "FG_ERR_DOMAIN", -6: "FG_ERR_NUMERIC"}
FG_SVK, FG_NEOHOOKE = 0, 1
FG_FP64, FG_MIXED = 0, 1
OP_MECH, OP_PFF, OP_PFF_PREC, OP_CHEM, OP_GRES = 0, 1, 2, 3, 4
FIELD_C, FIELD_F, FIELD_D, FIELD_H, FIELD_P = 0, 1, 2, 3, 4
SITES = {0: "mech.xfwd_tangent", 1: "mech.yfwd", 2: "mech.z_project", 3: "mech.yinv",
         4: "mech.xinv_dot", 5: "mech.cg_update"}


class FgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double)]


class Phase(C.Structure):
    _fields_ = [("law", C.c_int), ("E", C.c_double), ("nu", C.c_double), ("Omega", C.c_double),
                ("c0", C.c_double), ("D", C.c_double), ("sigma_max", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("gc", C.c_double), ("lc", C.c_double),
                ("RT", C.c_double), ("cmax", C.c_double), ("tol_newton", C.c_double),
                ("tol_cg", C.c_double), ("tol_chem", C.c_double), ("tol_chem_cg", C.c_double),
                ("tol_pff_cg", C.c_double), ("tol_stag", C.c_double), ("cg_forcing", C.c_double),
                ("max_newton", C.c_int), ("max_cg", C.c_int), ("max_chem_newton", C.c_int),
                ("max_stag", C.c_int), ("cuda_stream", C.c_void_p), ("l2_fraction", C.c_double),
                ("cg_indefinite", C.c_int), ("chem_full_jacobian", C.c_int),
                ("l2_prefetch", C.c_int), ("residual_ff", C.c_int), ("z_columns", C.c_int),
                ("cluster_pass", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("newton_chem", C.c_int), ("newton_mech", C.c_int), ("cg_chem", C.c_int),
                ("cg_mech", C.c_int), ("cg_pff", C.c_int), ("stag", C.c_int),
                ("inner_refine", C.c_int), ("cg_truncated", C.c_int), ("newton_damped", C.c_int),
                ("cg_negcurv", C.c_int), ("newton_shifted", C.c_int), ("newton_minres", C.c_int),
                ("cg_graph_replays", C.c_int),
                ("err_mech", C.c_double), ("err_chem", C.c_double),
                ("mass", C.c_double), ("mass_err", C.c_double), ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AdjStats(C.Structure):
    _fields_ = [("steps", C.c_int), ("recomputed", C.c_int), ("sweeps", C.c_int),
                ("gmres", C.c_int), ("cg_mech", C.c_int), ("cg_pff", C.c_int), ("cg_chem", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


FG_LOSS_CRACK_ENERGY = 0
FG_LOSS_SEEDS = 1

EXPORTS = ["fg_default_opts", "fg_supported_size", "fg_setup", "fg_step", "fg_residual",
           "fg_apply", "fg_get_field", "fg_set_field", "fg_time_apply", "fg_profile",
           "fg_profile_read", "fg_mech_apply_noalloc", "fg_batch_setup", "fg_batch_step",
           "fg_batch_apply", "fg_batch_time_apply", "fg_batch_destroy", "fg_autotune", "fg_autotune_report", "fg_solve_mech", "fg_adjoint_mech",
           "fg_tape_begin", "fg_adjoint", "fg_save", "fg_load", "fg_set_stress_control",
           "fg_displacement", "fg_displacement_adjoint", "fg_kernel_launches", "fg_destroy",
           "fg_last_error"]

_libs = {}


def load_library(path=LIB_PATH):
    """Loads a build of the C ABI and declares its signatures."""
    path = os.path.abspath(path)
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built: run __graft_entry__.build()")
    lib = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    lib.fg_default_opts.argtypes = [C.POINTER(Opts)]
    lib.fg_default_opts.restype = None
    lib.fg_supported_size.argtypes = [C.c_int]
    lib.fg_setup.argtypes = [C.POINTER(C.c_void_p), C.POINTER(Grid), C.POINTER(Phase), C.c_int,
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_void_p, C.POINTER(Opts)]
    lib.fg_step.argtypes = [C.c_void_p, C.c_double, dp, C.POINTER(Stats)]
    lib.fg_residual.argtypes = [C.c_void_p, dp, dp, dp]
    lib.fg_apply.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double, dp]
    lib.fg_get_field.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int]
    lib.fg_set_field.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int]
    lib.fg_time_apply.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, dp]
    lib.fg_profile.argtypes = [C.c_void_p, C.c_int, C.c_int]
    lib.fg_profile_read.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), dp, dp]
    lib.fg_mech_apply_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                          C.c_double] + [C.c_void_p] * 9 + [dp, C.c_void_p]
    lib.fg_autotune.argtypes = [C.c_void_p, dp]
    lib.fg_autotune_report.argtypes = [C.c_void_p, C.POINTER(C.c_int), dp]
    lib.fg_solve_mech.argtypes = [C.c_void_p, dp, C.POINTER(Stats)]
    lib.fg_adjoint_mech.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]
    lib.fg_tape_begin.argtypes = [C.c_void_p, C.c_int]
    lib.fg_displacement.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    lib.fg_displacement_adjoint.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    lib.fg_save.argtypes = [C.c_void_p, C.c_char_p]
    lib.fg_set_stress_control.argtypes = [C.c_void_p, C.c_int, dp]
    lib.fg_load.argtypes = [C.c_void_p, C.c_char_p]
    lib.fg_adjoint.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, dp,
                               C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(AdjStats)]
    lib.fg_batch_setup.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p)]
    lib.fg_batch_step.argtypes = [C.c_void_p, C.c_double, dp, C.POINTER(Stats)]
    lib.fg_batch_apply.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_void_p)]
    lib.fg_batch_time_apply.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, C.POINTER(C.c_int)]
    lib.fg_batch_destroy.argtypes = [C.c_void_p]
    lib.fg_batch_destroy.restype = None
    lib.fg_kernel_launches.restype = C.c_longlong
    lib.fg_destroy.argtypes = [C.c_void_p]
    lib.fg_destroy.restype = None
    lib.fg_last_error.restype = C.c_char_p
    _libs[path] = lib
    return lib


def kernel_launches(lib=None):
    return int((lib or load_library()).fg_kernel_launches())


def default_opts(lib=None):
    lib = lib or load_library()
    o = Opts()
    lib.fg_default_opts(C.byref(o))
    return o


def _ptr(a):
    """Address of a numpy array or a torch tensor."""
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _on_device(a):
    """True for a CUDA torch tensor (passed to the library as a device pointer)."""
    return hasattr(a, "data_ptr") and bool(getattr(a, "is_cuda", False))


def _dev64(a):
    """A CUDA tensor as the library expects it: float64, contiguous."""
    import torch
    if a.dtype != torch.float64 or not a.is_contiguous():
        a = a.to(torch.float64).contiguous()
    return a


def _arg64(a):
    """Host numpy float64 copy, or the CUDA tensor itself (float64, contiguous)."""
    return _dev64(a) if _on_device(a) else _f64(a).ravel()


def _out64(shape, like):
    """An output buffer of float64: a CUDA tensor on like's device when like is one, else
    a numpy array."""
    if like is not None and _on_device(like):
        import torch
        return torch.empty(shape, dtype=torch.float64, device=like.device)
    return np.empty(shape)


class Solver:
    """One periodic RVE: owns an ``fg_ctx``.  Host arrays are numpy, (nz, ny, nx)."""

    def __init__(self, shape, h, phases, phase_id, cdot_B, c_init=None, log_E=None, log_D=None,
                 log_gc=None, log_smax=None, opts=None, precision=FG_FP64, stream=None, lib=None,
                 **opt_kw):
        self.lib = lib or load_library()
        nz, ny, nx = shape
        self.shape = tuple(shape)
        self.h = tuple(float(x) for x in h)
        self.V = nx * ny * nz
        g = Grid(nx, ny, nz, *[float(x) for x in h])
        ph = (Phase * len(phases))()
        for k, p in enumerate(phases):
            ph[k] = Phase(int(p.law), p.E, p.nu, p.Omega, p.c0, p.D, p.sigma_max)
        o = opts or default_opts(self.lib)
        o.precision = precision
        for k, v in opt_kw.items():
            setattr(o, k, v)
        if stream is not None:
            o.cuda_stream = C.c_void_p(stream)
        self.opts = o
        self._keep = [np.ascontiguousarray(phase_id, dtype=np.uint8).ravel(), _f64(cdot_B).ravel()]
        opt_arrays = []
        for a in (c_init, log_E, log_D, log_gc, log_smax):
            opt_arrays.append(None if a is None else _f64(a).ravel())
        self._keep += opt_arrays
        ctx = C.c_void_p()
        rc = self.lib.fg_setup(C.byref(ctx), C.byref(g), ph, len(phases), _ptr(self._keep[0]),
                               _ptr(self._keep[1]),
                               *[None if a is None else _ptr(a) for a in opt_arrays],
                               C.byref(o))
        self._check(rc)
        self.ctx = ctx

    def _check(self, rc):
        if rc != FG_OK:
            raise FgError(rc, self.lib.fg_last_error().decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.fg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, dt, Fbar=None, check=True):
        Fb = _f64(np.eye(3) if Fbar is None else Fbar).ravel()
        st = Stats()
        rc = self.lib.fg_step(self.ctx, dt, Fb.ctypes.data_as(C.POINTER(C.c_double)), C.byref(st))
        if check:
            self._check(rc)
        return st.as_dict()

    def residual(self):
        em, ec, ms = C.c_double(), C.c_double(), C.c_double()
        self._check(self.lib.fg_residual(self.ctx, C.byref(em), C.byref(ec), C.byref(ms)))
        return em.value, ec.value, ms.value

    def get(self, field, device=None):
        """A field as a numpy array, or (device given, e.g. "cuda") as a CUDA tensor copied
        on the device."""
        n = 9 if field in (FIELD_F, FIELD_P) else 1
        shp = (3, 3) + self.shape if n == 9 else self.shape
        if device is not None:
            import torch
            out = torch.empty(shp, dtype=torch.float64, device=device)
            self._check(self.lib.fg_get_field(self.ctx, field, _ptr(out), 1))
            return out
        out = np.empty(shp)
        self._check(self.lib.fg_get_field(self.ctx, field, _ptr(out), 0))
        return out

    def set(self, field, value):
        """Overwrites a stored field from a host array or a CUDA tensor."""
        v = _arg64(value)
        self._check(self.lib.fg_set_field(self.ctx, field, _ptr(v), int(_on_device(v))))

    def apply(self, op, x, y, prec=0, dt=1.0):
        """y = op(x) on device buffers (torch tensors); returns <x, y>."""
        dot = C.c_double()
        self._check(self.lib.fg_apply(self.ctx, op, prec, _ptr(x), _ptr(y), dt, C.byref(dot)))
        return dot.value

    def profile(self, site, enable=True):
        self._check(self.lib.fg_profile(self.ctx, site, int(enable)))

    def profile_read(self, site):
        """(launches, total ms, full volumes covered) of a profiled launch site."""
        n, ms, vol = C.c_int(), C.c_double(), C.c_double()
        self._check(self.lib.fg_profile_read(self.ctx, site, C.byref(n), C.byref(ms), C.byref(vol)))
        return n.value, ms.value, vol.value

    def solve_mech(self, Fbar=None, check=True):
        Fb = _f64(np.eye(3) if Fbar is None else Fbar).ravel()
        st = Stats()
        rc = self.lib.fg_solve_mech(self.ctx, Fb.ctypes.data_as(C.POINTER(C.c_double)), C.byref(st))
        if check:
            self._check(rc)
        return st.as_dict()

    def adjoint_mech(self, W):
        """dL/dlogE for a loss with dL/dF = W (host array (3, 3, ...) or CUDA tensor; the
        gradient comes back the same way)."""
        Wh = _arg64(W)
        g = _out64(self.shape, Wh)
        it = C.c_int()
        self._check(self.lib.fg_adjoint_mech(self.ctx, _ptr(Wh), _ptr(g), C.byref(it)))
        return g, it.value

    def stress_control(self, mask, Pbar=None):
        """Mixed macroscopic control: mask (3, 3) bool of stress-controlled components with
        prescribed mean stress Pbar (3, 3); None or an all-False mask: strain control."""
        m = 0 if mask is None else int(sum(1 << k for k, on in enumerate(np.asarray(mask).ravel()) if on))
        Pb = _f64(np.zeros(9) if Pbar is None else Pbar).ravel()
        self._check(self.lib.fg_set_stress_control(self.ctx, m, Pb.ctypes.data_as(C.POINTER(C.c_double))))

    def save(self, path):
        """Writes the evolving state to a restart file (fg_save)."""
        self._check(self.lib.fg_save(self.ctx, os.fsencode(path)))

    def load(self, path):
        """Reads a restart file written for the same grid, law and materials (fg_load)."""
        self._check(self.lib.fg_load(self.ctx, os.fsencode(path)))

    def tape(self, ckpt_every=1):
        """Starts recording the following steps for ``adjoint`` (checkpoint every k steps)."""
        self._check(self.lib.fg_tape_begin(self.ctx, int(ckpt_every)))

    def adjoint(self, loss=FG_LOSS_CRACK_ENERGY, seed_c=None, seed_F=None, seed_d=None):
        """Reverse of the recorded steps: returns (loss value, dict(E, gc, D) of per-voxel
        dL/dlog E, dL/dlog g_c, dL/dlog D, statistics)."""
        seeds = [None if a is None else _arg64(a) for a in (seed_c, seed_F, seed_d)]
        like = next((a for a in seeds if a is not None), None)
        g = {k: _out64(self.shape, like) for k in ("E", "gc", "D")}
        val = C.c_double()
        st = AdjStats()
        self._check(self.lib.fg_adjoint(self.ctx, int(loss),
                                        *[None if a is None else _ptr(a) for a in seeds],
                                        C.byref(val), _ptr(g["E"]), _ptr(g["gc"]), _ptr(g["D"]),
                                        C.byref(st)))
        return val.value, g, st.as_dict()

    def displacement(self, F=None, Fbar=None):
        """Displacement (3, nz, ny, nx) at the voxel corners of F and Fbar (both None: the
        current state): (Fbar - I) x + u~ with grad u~ = F - Fbar (fg_displacement)."""
        if (F is None) != (Fbar is None):
            raise ValueError("F and Fbar are given together")
        Fa = None if F is None else _arg64(F)
        Fb = None if Fbar is None else _f64(Fbar).ravel()
        u = _out64((3,) + self.shape, Fa)
        self._check(self.lib.fg_displacement(self.ctx, None if Fa is None else _ptr(Fa),
                                             None if Fb is None else _ptr(Fb), _ptr(u),
                                             int(_on_device(u))))
        return u

    def displacement_adjoint(self, r):
        """(du~/dF)^T r for r (3, nz, ny, nx): a (3, 3, nz, ny, nx) field
        (fg_displacement_adjoint)."""
        ra = _arg64(r)
        g = _out64((3, 3) + self.shape, ra)
        self._check(self.lib.fg_displacement_adjoint(self.ctx, _ptr(ra), _ptr(g),
                                                     int(_on_device(g))))
        return g

    def autotune(self):
        ms = C.c_double()
        self._check(self.lib.fg_autotune(self.ctx, C.byref(ms)))
        return ms.value

    def autotune_report(self):
        """Choices in force (kx planes per chunk, one-component X-inv update, L2 prefetch,
        columns per block of the FP32 projection pass) and the autotuner's X-inv update
        times [prefetch off/on][nine/one component]."""
        ch = (C.c_int * 5)()
        ms = (C.c_double * 4)()
        self._check(self.lib.fg_autotune_report(self.ctx, ch, ms))
        return {"kx_chunk": ch[0], "xinv_per_component": ch[1], "l2_prefetch": ch[2],
                "z_proj_columns_per_block": ch[3], "cluster_yzy_mech": ch[4] & 1,
                "cluster_yzy_chem": (ch[4] >> 1) & 1,
                "xinv_ms": {"nine": ms[0], "one": ms[1], "nine_prefetch": ms[2],
                            "one_prefetch": ms[3]}}

    def time_apply(self, op, prec, n):
        ms = C.c_double()
        self._check(self.lib.fg_time_apply(self.ctx, op, prec, n, C.byref(ms)))
        return ms.value


class Batch:
    """Independent RVEs stepped together (fg_batch_*); members are ``Solver`` objects."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.lib = self.solvers[0].lib
        arr = (C.c_void_p * len(self.solvers))(*[s.ctx for s in self.solvers])
        h = C.c_void_p()
        rc = self.lib.fg_batch_setup(C.byref(h), len(self.solvers), arr)
        if rc != FG_OK:
            raise FgError(rc, self.lib.fg_last_error().decode())
        self.h = h

    def step(self, dt, Fbar=None, check=True):
        Fb = _f64(np.eye(3) if Fbar is None else Fbar).ravel()
        st = (Stats * len(self.solvers))()
        rc = self.lib.fg_batch_step(self.h, dt, Fb.ctypes.data_as(C.POINTER(C.c_double)), st)
        if check and rc != FG_OK:
            raise FgError(rc, self.lib.fg_last_error().decode())
        return [s.as_dict() for s in st]

    def apply(self, xs, ys, prec=0, op=None):
        """y_i = A_i x_i for every member (OP_MECH) in grouped launches: xs, ys are one
        buffer per member (torch tensors on the device; numpy arrays with the emulation)."""
        op = OP_MECH if op is None else op
        n = len(self.solvers)
        if len(xs) != n or len(ys) != n:
            raise ValueError("one input and one output per member")
        xa = (C.c_void_p * n)(*[_ptr(x) for x in xs])
        ya = (C.c_void_p * n)(*[_ptr(y) for y in ys])
        rc = self.lib.fg_batch_apply(self.h, op, prec, xa, ya)
        if rc != FG_OK:
            raise FgError(rc, self.lib.fg_last_error().decode())

    def time_apply(self, prec=1, n=20):
        """Milliseconds per application of every member's mechanical operator: grouped
        launches replayed from a CUDA graph, grouped launches, members one by one on one
        stream, members on their own streams; and (groups, launches per grouped
        application, launches per one-by-one application)."""
        ms = (C.c_double * 4)()
        info = (C.c_int * 3)()
        rc = self.lib.fg_batch_time_apply(self.h, prec, n, ms, info)
        if rc != FG_OK:
            raise FgError(rc, self.lib.fg_last_error().decode())
        return list(ms), list(info)

    def close(self):
        if getattr(self, "h", None):
            self.lib.fg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_workload(w, precision=FG_FP64, lib=None, stream=None, **opt_kw):
    """Solver for a ``synth.Workload``."""
    kw = dict(w.tol)
    kw.update(opt_kw)
    return Solver(w.shape, w.h, w.phases, w.phase_id, w.cdot_B, c_init=w.c_init, log_E=w.log_E,
                  log_D=w.log_D, log_gc=w.log_gc, log_smax=w.log_smax, precision=precision,
                  lib=lib, stream=stream,
                  gc=w.gc, lc=w.lc,
                  RT=w.RT, cmax=w.cmax, **kw)
