"""Seeded synthetic workloads shaped like the paper's particle problems.

This module only *generates inputs*: voxel phase maps, the influx source field, the
initial concentration and optional per-voxel log-scale fields, plus the material
constants and solver tolerances of each workload.  It holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

Geometry follows the paper's set-up: one active particle embedded in a compliant,
almost non-diffusive buffer phase that emulates the surrounding electrolyte
(Sec. 4.3, Sec. 5.1), with the ion influx imposed as a volume source in a band of
width dL just inside the particle surface (Eqs. neumann1, neumann2).  All random
numbers come from ``numpy.random.Generator(PCG64(seed))``.

Workloads (sizes in voxels, voxel size h = 0.1 um unless stated):

* ``disc2d``    64x64x1 plane strain, disc radius 20, band 6 voxels, 10 steps.
* ``ellipsoid`` 128^3, semi-axes 50/40/35 with a Gaussian-filtered rough surface
  (std 1.5 voxels, correlation length 4 voxels), band 8 voxels, 50 steps.
* ``ellipsoid`` at 256^3 scaled x2 (semi-axes 100/80/70, roughness std 3,
  correlation 8) plus a smooth Gaussian concentration perturbation of std 0.02
  (correlation 8 voxels) around c = 0.07 inside the particle (its stress-free
  concentration), 100 steps.
* ``spheres``   64 RVEs with edge N in {48, 64, 80, 96} and sphere radius
  U(0.30, 0.45) N.
* ``ellipsoid`` 128^3 with per-voxel log E, log g_c, log D ~ N(0, 0.1^2).
* ``multi_particle`` several non-overlapping rough ellipsoids in one RVE.
* ``gumbel_disc`` 512^2 Saint-Venant-Kirchhoff disc with Weibull-type random stiffness and
  strength and the paper's Omega = 1.3 (Sec. 5.1).
* ``plate``     64x64x1 Saint-Venant-Kirchhoff plate of Sec. 4.3 with a stronger influx
  at one corner.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LAW_SVK = 0
LAW_NEOHOOKE = 1
PARTICLE = 0
BUFFER = 1


@dataclass
class PhaseSpec:
    law: int = LAW_NEOHOOKE
    E: float = 10e9
    nu: float = 0.3
    Omega: float = 0.0
    c0: float = 0.01
    D: float = 1e-14
    sigma_max: float = 100e6


@dataclass
class Workload:
    name: str
    shape: tuple                 # (nz, ny, nx)
    h: tuple                     # (hx, hy, hz) in m
    phases: list                 # [PhaseSpec(particle), PhaseSpec(buffer)]
    phase_id: np.ndarray         # uint8 (nz, ny, nx)
    cdot_B: np.ndarray           # float64 (nz, ny, nx), 1/s
    c_init: np.ndarray           # float64 (nz, ny, nx)
    gc: float                    # J/m^2
    lc: float                    # m
    dt: float                    # s
    nsteps: int
    log_E: np.ndarray | None = None
    log_gc: np.ndarray | None = None
    log_D: np.ndarray | None = None
    log_smax: np.ndarray | None = None
    RT: float = 8.314462618 * 298.15
    cmax: float = 3.0e4
    tol: dict = field(default_factory=lambda: dict(
        tol_newton=1e-9, tol_cg=1e-10, tol_chem=1e-9, tol_chem_cg=1e-10, tol_pff_cg=1e-10,
        tol_stag=1e-9, max_newton=30, max_cg=5000, max_chem_newton=50, max_stag=50))

    @property
    def nvox(self):
        return int(np.prod(self.shape))


def default_phases(E=10e9, nu=0.3, c0=0.01, D=1e-14, sigma_max=100e6, vol_change=0.10,
                   buffer_E=1e-3, buffer_D=1e-5, law=LAW_NEOHOOKE):
    """Particle and buffer constants.  The swelling coefficient gives ``vol_change`` of
    volume change at c = 1 relative to the stress-free c0: Omega = vol_change/(1-c0)."""
    omega = vol_change / (1.0 - c0)
    particle = PhaseSpec(law=law, E=E, nu=nu, Omega=omega, c0=c0, D=D, sigma_max=sigma_max)
    buffer = PhaseSpec(law=law, E=E * buffer_E, nu=nu, Omega=0.0, c0=c0, D=D * buffer_D,
                       sigma_max=sigma_max)
    return [particle, buffer]


def _grid_coords(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cz, cy, cx = (nz - 1) / 2.0, (ny - 1) / 2.0, (nx - 1) / 2.0
    return x - cx, y - cy, z - cz


def influx_band(particle, width):
    """Particle voxels whose Euclidean distance to the nearest buffer voxel is <= width."""
    from scipy import ndimage
    if particle.shape[0] == 1:
        dist = ndimage.distance_transform_edt(particle[0])[None]
    else:
        dist = ndimage.distance_transform_edt(particle)
    return particle & (dist <= width)


def _rough_field(rng, shape, std, corr):
    from scipy import ndimage
    noise = rng.standard_normal(shape)
    sm = ndimage.gaussian_filter(noise, sigma=corr, mode="wrap")
    sd = sm.std()
    return sm * (std / sd) if sd > 0 else sm


def _finish(name, shape, h, particle, band_width, nsteps, dt, rng, phases=None, c_perturb=0.0,
            target_c=0.5, gc=1.0, lc_vox=2.0, perturb_corr=8.0, perturb_mean=0.07):
    phases = phases or default_phases()
    phase_id = np.where(particle, PARTICLE, BUFFER).astype(np.uint8)
    band = influx_band(particle, band_width)
    c0 = phases[PARTICLE].c0
    # influx rate: the band alone would reach target_c at the last step without diffusion
    rate = (target_c - c0) / (dt * nsteps)
    cdot_B = np.where(band, rate, 0.0)
    c_init = np.full(shape, c0)
    if c_perturb > 0.0:
        # smooth Gaussian random field of standard deviation c_perturb (correlation length
        # perturb_corr voxels) around perturb_mean inside the particle, whose stress-free
        # concentration is set to that mean: only the fluctuation is an eigenstrain at t = 0
        pert = _rough_field(rng, shape, c_perturb, perturb_corr)
        c_init = np.where(particle, np.clip(perturb_mean + pert, 0.005, 0.995), c0)
        p = phases[PARTICLE]
        phases = [PhaseSpec(law=p.law, E=p.E, nu=p.nu, Omega=p.Omega, c0=perturb_mean, D=p.D,
                            sigma_max=p.sigma_max)] + list(phases[1:])
    return Workload(name=name, shape=shape, h=h, phases=phases, phase_id=phase_id,
                    cdot_B=cdot_B, c_init=c_init, gc=gc, lc=lc_vox * h[0], dt=dt, nsteps=nsteps)


def disc2d(n=64, radius=20.0, band=6, nsteps=10, seed=0, h=0.1e-6, **kw):
    """2D plane-strain disc particle in a buffer matrix (configuration of Sec. 5.1 type)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (1, n, n)
    x, y, _ = _grid_coords(shape)
    particle = (x * x + y * y) <= radius * radius
    return _finish("disc2d", shape, (h, h, h), particle, band, nsteps, 1.0, rng, **kw)


def ellipsoid(n=128, axes=(50.0, 40.0, 35.0), rough_std=1.5, rough_corr=4.0, band=8,
              nsteps=50, seed=0, h=0.1e-6, c_perturb=0.0, shape=None, **kw):
    """3D ellipsoidal particle with a seeded rough surface: voxel x is particle when
    (rho(x) - 1) R_min <= eta(x), rho the ellipsoidal radius and eta the roughness."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = shape or (n, n, n)
    x, y, z = _grid_coords(shape)
    a, b, c = axes
    rho = np.sqrt((x / a) ** 2 + (y / b) ** 2 + (z / c) ** 2)
    eta = _rough_field(rng, shape, rough_std, rough_corr) if rough_std > 0 else 0.0
    particle = (rho - 1.0) * min(axes) <= eta
    return _finish("ellipsoid", shape, (h, h, h), particle, band, nsteps, 1.0, rng,
                   c_perturb=c_perturb, **kw)


def multi_particle(n=128, count=4, rmin=0.12, rmax=0.2, rough_std=1.0, rough_corr=3.0, band=4,
                   nsteps=50, seed=0, h=0.1e-6, **kw):
    """Several rough ellipsoidal particles in one periodic RVE (a piece of electrode, as in
    the paper's outlook): semi-axes drawn from U(rmin, rmax) n, centres placed by rejection
    so that no two particles overlap (periodic distance), each with its own influx band."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n, n, n)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    eta = _rough_field(rng, shape, rough_std, rough_corr) if rough_std > 0 else 0.0
    particle = np.zeros(shape, dtype=bool)
    placed = []
    tries = 0
    while len(placed) < count:
        tries += 1
        if tries > 1000:
            raise ValueError("multi_particle: could not place the particles")
        ax = rng.uniform(rmin, rmax, size=3) * n
        ctr = rng.uniform(0, n, size=3)
        if any(np.linalg.norm(((ctr - c2 + n / 2) % n) - n / 2) < ax.max() + a2.max() + band
               for c2, a2 in placed):
            continue
        placed.append((ctr, ax))
        d = [((q - c + n / 2) % n) - n / 2 for q, c in zip((x, y, z), ctr)]
        rho = np.sqrt((d[0] / ax[0]) ** 2 + (d[1] / ax[1]) ** 2 + (d[2] / ax[2]) ** 2)
        particle |= (rho - 1.0) * ax.min() <= eta
    return _finish("multi_particle", shape, (h, h, h), particle, band, nsteps, 1.0, rng, **kw)


BENCH_BUFFER_E = 1e-2  # buffer stiffness of the benchmark particle, relative to the particle's


def ellipsoid256(seed=0, nsteps=100, **kw):
    """The 256^3 benchmark particle.  Its buffer is 100 times softer than the particle: with
    1000 times, the particle's rigid rotations against the buffer lose their stiffness to
    the compressive prestress after a few steps and the mechanical Newton stalls."""
    kw.setdefault("phases", default_phases(buffer_E=BENCH_BUFFER_E))
    return ellipsoid(n=256, axes=(100.0, 80.0, 70.0), rough_std=3.0, rough_corr=8.0, band=8,
                     nsteps=nsteps, seed=seed, c_perturb=0.02, **kw)


def sphere(n, radius_frac, band=4, nsteps=20, seed=0, h=0.1e-6, **kw):
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n, n, n)
    x, y, z = _grid_coords(shape)
    particle = (x * x + y * y + z * z) <= (radius_frac * n) ** 2
    return _finish("sphere", shape, (h, h, h), particle, band, nsteps, 1.0, rng, **kw)


def sphere_batch(count=64, sizes=(48, 64, 80, 96), rmin=0.30, rmax=0.45, nsteps=20, seed=0):
    """Independent particle RVEs of uneven size (one persistent batch)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.choice(np.array(sizes), size=count)
    rs = rng.uniform(rmin, rmax, size=count)
    return [sphere(int(n), float(r), nsteps=nsteps, seed=seed + 1 + i,
                   phases=default_phases(buffer_E=BENCH_BUFFER_E))
            for i, (n, r) in enumerate(zip(ns, rs))]


def gumbel_log_scale(rng, shape, m=3.0):
    """Per-voxel log-scale of a property drawn with the law of Eq. Gumbell,
    X_i = X log(1/(1 - w_i))^(1/m) with w_i ~ U(0, 1): returns log(X_i / X)."""
    om = rng.uniform(size=shape)
    return np.log(np.log(1.0 / (1.0 - om))) / m


def gumbel_disc(n=512, diameter_frac=0.8, band=6, nsteps=200, seed=0, m=3.0, h=16e-6 / 512,
                E=15e9, Omega=1.3, sigma_max=100e6, random_strength=True):
    """2D circular Saint-Venant-Kirchhoff particle with Weibull-type random stiffness
    (Sec. 5.1, Eq. Gumbell): E_i = E log(1/(1 - w_i))^(1/m), w_i ~ U(0, 1), m = 3, carried
    as the per-voxel log-stiffness log_E = log(log(1/(1 - w_i)))/m, and the paper's
    swelling Omega = 1.3.  The strength sigma_max (100 MPa in the text of Sec. 5.1) is
    drawn per voxel from the same law with its own w_i (log_smax; random_strength=False
    keeps it uniform).  With E = 15 GPa and Omega = 1.3 the elastic chemical potential
    reaches several RT, where the Newton of Alg. 3 (Jacobian of the ideal part only) stops
    converging; the workload therefore runs the chemistry Newton with the full Jacobian
    (chem_full_jacobian).  The influx fills the particle to a mean c of 0.5 over nsteps
    steps.  The default of 200 keeps the first step free of damage, as in Sec. 5.1: at
    512^2 with 20 steps the first step already cracked most of the particle and needed
    341 staggered iterations, so the staggered cap is raised to 400 (max_stag)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (1, n, n)
    x, y, _ = _grid_coords(shape)
    particle = (x * x + y * y) <= (0.5 * diameter_frac * n) ** 2
    c0 = 0.01
    phases = default_phases(E=E, c0=c0, law=LAW_SVK, vol_change=Omega * (1.0 - c0), buffer_E=1e-5,
                            sigma_max=sigma_max)
    w = _finish("gumbel_disc", shape, (h, h, h), particle, band, nsteps, 1.0, rng, phases=phases)
    w.log_E = np.where(particle, gumbel_log_scale(rng, shape, m), 0.0)
    if random_strength:
        w.log_smax = np.where(particle, gumbel_log_scale(rng, shape, m), 0.0)
    w.tol = dict(w.tol, chem_full_jacobian=1, max_stag=400)
    return w


def plate(n=64, plate_frac=0.75, nsteps=20, corner_ratio=1.5, corner_frac=0.25, seed=0):
    """The chemo-mechanical fracture plate of Sec. 4.3 (Table tab:4.3_properties): a square
    Saint-Venant-Kirchhoff plate, E = 15 GPa, nu = 0.3, sigma_max = 50 MPa, Omega = 1.3,
    g_c = 2 J/m^2, l_c = 2 voxels, D = 1e-15 m^2/s, in a buffer 1e-5 times as stiff and as
    diffusive, on an n x n x 1 grid of side 8 um (h = 0.125 um for n = 64, so that l_c is
    the table's 0.25 um).  The influx enters through a band one voxel wide along the plate's
    edges (dL = 1 voxel); the band voxels within corner_frac of the edge length of the
    (+x, +y) corner take corner_ratio times the edge rate (the table's 3e-4 against
    2e-4), which breaks the plate's symmetry so that the crack starts there.  The plate
    occupies the central plate_frac of each in-plane axis (the buffer's size is only drawn
    in the paper).  The edge rate fills the plate to a mean c of 0.5 over nsteps steps of
    dt = h^2/D (Fourier number 1); like the Sec. 5.1 disc with Omega = 1.3, the chemistry
    Newton runs with the full Jacobian.  With these readings the plate cracks along its
    edges in step 3 (d near 1 in 836 voxels)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (1, n, n)
    h = 8e-6 / n
    x, y, _ = _grid_coords(shape)
    half = 0.5 * plate_frac * n
    particle = (np.abs(x) < half) & (np.abs(y) < half)
    c0 = 0.01
    D = 1e-15
    phases = default_phases(E=15e9, nu=0.3, c0=c0, D=D, sigma_max=50e6, law=LAW_SVK,
                            vol_change=1.3 * (1.0 - c0), buffer_E=1e-5, buffer_D=1e-5)
    dt = h * h / D
    w = _finish("plate", shape, (h, h, h), particle, 1, nsteps, dt, rng, phases=phases,
                gc=2.0)
    corner = (x > half - 2.0 * corner_frac * half) & (y > half - 2.0 * corner_frac * half)
    w.cdot_B = np.where(corner, corner_ratio * w.cdot_B, w.cdot_B)
    # the cracked plate's mechanics is nearly singular (stiffness (1 - d)^2 ~ 1e-7 in the
    # crack): Krylov solves there may need more than the default 5000 iterations
    w.tol = dict(w.tol, chem_full_jacobian=1, max_stag=400, max_cg=20000)
    return w


def with_log_fields(w, std=0.1, seed=0):
    """Attach per-voxel log-stiffness, log-toughness and log-diffusivity ~ N(0, std^2)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    w.log_E = rng.normal(0.0, std, size=w.shape)
    w.log_gc = rng.normal(0.0, std, size=w.shape)
    w.log_D = rng.normal(0.0, std, size=w.shape)
    return w


def random_state(shape, seed=0, f_amp=0.03, c_lo=0.05, c_hi=0.6, d_hi=0.5):
    """Random but physical fields for operator tests: F = I + small perturbation,
    c in (c_lo, c_hi), d in [0, d_hi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    F = np.zeros((3, 3) + tuple(shape))
    for i in range(3):
        F[i, i] = 1.0
    F = F + f_amp * rng.standard_normal(F.shape)
    if shape[0] == 1:  # plane strain: no out-of-plane shear
        F[0, 2] = F[1, 2] = F[2, 0] = F[2, 1] = 0.0
    c = rng.uniform(c_lo, c_hi, size=shape)
    d = rng.uniform(0.0, d_hi, size=shape)
    return F, c, d


def random_tensor_field(shape, seed=0, ncomp=9):
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    return rng.standard_normal((ncomp,) + tuple(shape))


def random_phase_map(shape, seed=0, frac=0.5):
    rng = np.random.Generator(np.random.PCG64(seed + 15485863))
    return (rng.uniform(size=shape) > frac).astype(np.uint8)
