"""The seeded input recipes of the synthetic workloads (CPU): influx band, influx rate,
the law of Eq. Gumbell, roughness and concentration perturbations, batch sizes and
determinism."""
import math

import numpy as np
import pytest

from paper_2411_16583_gb300 import synth as S


def test_influx_band_is_the_euclidean_band_inside_the_particle():
    """Band = particle voxels whose distance to the nearest buffer voxel is <= the width
    (Eqs. neumann1-2, band dL): on a disc of radius R it is the annulus R - width < r <= R,
    up to one voxel of discretisation."""
    w = S.disc2d(n=64, radius=20.0, band=6)
    x, y, _ = S._grid_coords(w.shape)
    r = np.sqrt(x * x + y * y)
    part = w.phase_id == S.PARTICLE
    band = w.cdot_B > 0
    assert np.all(part[band])
    assert not band[part & (r < 20.0 - 6.0 - 1.0)].any()
    assert band[part & (r > 20.0 - 6.0 + 1.0)].all()


def test_influx_rate_fills_the_particle_to_the_target_mean():
    """cdot_B = (0.5 - c0)/(dt n_steps) in the band and 0 elsewhere, so the band alone would
    reach c = 0.5 at the last step without diffusion."""
    w = S.disc2d(n=64, radius=20.0, band=6, nsteps=10)
    c0 = w.phases[S.PARTICLE].c0
    rate = (0.5 - c0) / (w.dt * w.nsteps)
    band = w.cdot_B > 0
    np.testing.assert_allclose(w.cdot_B[band], rate, rtol=1e-15)
    assert np.all(w.cdot_B[~band] == 0.0)


def test_gumbel_log_scale_follows_the_weibull_law():
    """X = log(1/(1 - w))^(1/m), w ~ U(0, 1) (Eq. Gumbell) has P(X <= x) = 1 - exp(-x^m):
    Kolmogorov-Smirnov against that law and the mean Gamma(1 + 1/m), for m = 3."""
    from scipy import stats
    rng = np.random.Generator(np.random.PCG64(11))
    x = np.exp(S.gumbel_log_scale(rng, (200000,), m=3.0))
    assert stats.kstest(x, lambda t: 1.0 - np.exp(-t ** 3.0)).pvalue > 1e-3
    assert abs(x.mean() - math.gamma(1.0 + 1.0 / 3.0)) < 5.0 * x.std() / math.sqrt(x.size)


def test_gumbel_disc_draws_stiffness_and_strength_independently():
    w = S.gumbel_disc(n=64, band=2)
    part = w.phase_id == S.PARTICLE
    assert w.log_smax is not None and w.log_E is not None
    assert np.all(w.log_E[~part] == 0.0) and np.all(w.log_smax[~part] == 0.0)
    rho = np.corrcoef(w.log_E[part], w.log_smax[part])[0, 1]
    assert abs(rho) < 5.0 / math.sqrt(part.sum())
    assert w.tol["max_stag"] == 400 and w.tol["chem_full_jacobian"] == 1
    assert S.gumbel_disc(n=64, band=2, random_strength=False).log_smax is None


def test_rough_ellipsoid_and_concentration_perturbation():
    """The rough surface is a Gaussian field rescaled to the requested std; the perturbed
    concentration is a smooth field of std 0.02 around 0.07 inside the particle, whose
    stress-free concentration is set to 0.07 (R17, R18)."""
    rng = np.random.Generator(np.random.PCG64(3))
    eta = S._rough_field(rng, (32, 32, 32), 1.5, 4.0)
    assert abs(eta.std() - 1.5) < 1e-12
    w = S.ellipsoid(n=64, axes=(25.0, 20.0, 17.5), rough_std=1.5, rough_corr=4.0, band=4,
                    c_perturb=0.02)
    part = w.phase_id == S.PARTICLE
    assert 0.05 < part.mean() < 0.25
    assert w.phases[S.PARTICLE].c0 == 0.07
    cp = w.c_init[part]
    assert abs(cp.mean() - 0.07) < 0.01 and 0.01 < cp.std() < 0.03
    assert np.all(w.c_init[~part] == w.phases[S.BUFFER].c0)


def test_sphere_batch_sizes_and_determinism():
    ws = S.sphere_batch(count=8)
    assert all(w.shape[0] in (48, 64, 80, 96) and w.shape[0] == w.shape[1] == w.shape[2]
               for w in ws)
    for w in ws:
        frac = (w.phase_id == S.PARTICLE).mean()
        assert 4.0 / 3.0 * math.pi * 0.29 ** 3 < frac < 4.0 / 3.0 * math.pi * 0.46 ** 3
    again = S.sphere_batch(count=8)
    for a, b in zip(ws, again):
        np.testing.assert_array_equal(a.phase_id, b.phase_id)
        np.testing.assert_array_equal(a.cdot_B, b.cdot_B)


@pytest.mark.parametrize("make", [lambda: S.disc2d(n=32, radius=10.0, band=2),
                                  lambda: S.multi_particle(n=32, count=2, band=2),
                                  lambda: S.gumbel_disc(n=32, band=2)])
def test_workloads_are_deterministic(make):
    a, b = make(), make()
    for f in ("phase_id", "cdot_B", "c_init", "log_E", "log_smax"):
        x, y = getattr(a, f), getattr(b, f)
        if x is None:
            assert y is None
        else:
            np.testing.assert_array_equal(x, y)
