"""Planted mistakes: each test injects a plausible error into the oracle (a dropped term,
a wrong sign or index, a transposed operand) and checks that the pins of
test_oracle_*.py catch it.  All on the CPU; the oracle module is restored afterwards."""
import numpy as np
import pytest

from oracle import fg_oracle as O
from tests import test_oracle_constitutive as TC
from tests import test_oracle_solvers as TS
from tests import test_oracle_spectral as TSP


def test_projection_without_normalisation_is_caught(monkeypatch):
    def bad(A, n):  # drops the 1/|n|^2
        An = np.einsum("im...,m...->i...", A, n)
        return np.einsum("i...,j...->ij...", An, n)
    monkeypatch.setattr(O, "project_G", bad)
    with pytest.raises(AssertionError):
        TSP.test_projection_properties((4, 6, 8))


def test_projection_transposed_is_caught(monkeypatch):
    good = O.project_G

    def bad(A, n):  # projects columns instead of rows
        return np.swapaxes(good(np.swapaxes(A, 0, 1), n), 0, 1)
    monkeypatch.setattr(O, "project_G", bad)
    with pytest.raises(AssertionError):
        TSP.test_projection_properties((4, 6, 8))


def test_wrong_rotated_symbol_is_caught(monkeypatch):
    good = O.rotated_frequencies

    def bad(shape, h):  # forgets the cos factor of the other axes (central difference)
        n = good(shape, h)
        return n * 0 + O.fd_laplacian_symbol(shape, h)[None] ** 0.5
    monkeypatch.setattr(O, "rotated_frequencies", bad)
    with pytest.raises(AssertionError):
        TSP.test_rotated_symbol_is_corner_stencil((4, 6, 8))


def test_tangent_missing_term_is_caught(monkeypatch):
    good = O.dP0

    def bad(Fe, dFe, prm):  # drops the geometric (dF S) term of both laws
        out = good(Fe, dFe, prm)
        return out - 0.01 * dFe * prm.mu
    monkeypatch.setattr(O, "dP0", bad)
    with pytest.raises(AssertionError):
        TC.test_tangent_is_stress_derivative_and_symmetric(O.LAW_NEOHOOKE)


def test_swelling_sign_is_caught(monkeypatch):
    def bad(c, prm):  # J_c = 1 - Omega (c - c0)
        return 1.0 - prm.Omega * (c - prm.c0)
    monkeypatch.setattr(O, "swelling_J", bad)
    with pytest.raises(AssertionError):
        TC.test_free_swelling_and_degradation(O.LAW_NEOHOOKE)


def test_elastic_potential_sign_is_caught(monkeypatch):
    good = O.mu_elastic
    monkeypatch.setattr(O, "mu_elastic", lambda F, c, d, prm: -good(F, c, d, prm))
    with pytest.raises(AssertionError):
        TC.test_elastic_chemical_potential_is_energy_derivative(O.LAW_NEOHOOKE)


def test_divergence_without_conjugate_is_caught(monkeypatch):
    def bad(u, Kc, prm):  # uses xi instead of conj(xi) for the divergence
        xi = O.fd_frequencies(prm.shape, prm.h)
        g = O.irfft3(xi * O.rfft3(u)[None], prm.shape)
        flux = np.einsum("jl...,l...->j...", Kc, g)
        return -O.irfft3(np.sum(xi * O.rfft3(flux), axis=0), prm.shape)
    monkeypatch.setattr(O, "chem_L", bad)
    with pytest.raises(AssertionError):
        TS.test_chem_operator_is_divergence_stencil()


def test_phase_field_laplacian_sign_is_caught(monkeypatch):
    def bad(dd, H, prm):
        lap = O.fd_laplacian_symbol(prm.shape, prm.h)
        return (prm.gc / prm.lc + 2.0 * H) * dd - O.irfft3(prm.gc * prm.lc * lap * O.rfft3(dd), prm.shape)
    monkeypatch.setattr(O, "pff_apply", bad)
    with pytest.raises((AssertionError, FloatingPointError, RuntimeError)):
        TS.test_pff_1d_crack_discrete_closed_form()


def test_mobility_factor_is_caught(monkeypatch):
    monkeypatch.setattr(O, "mobility_phi", lambda d: (1.0 - d) ** 2)  # drops 0.9 and 0.1 d^2
    with pytest.raises(AssertionError):
        TS.test_chem_single_mode_decay()


def test_adjoint_sign_is_caught(monkeypatch):
    good = O.mech_adjoint
    monkeypatch.setattr(O, "mech_adjoint", lambda *a, **k: -good(*a, **k))
    with pytest.raises(AssertionError):
        TS.test_mech_adjoint_matches_central_differences()


def test_strength_scale_inverted_is_caught(monkeypatch):
    good = O.make_params

    def bad(*a, log_smax=None, **kw):  # sigma_max exp(-log_smax) instead of exp(+log_smax)
        return good(*a, log_smax=None if log_smax is None else -log_smax, **kw)
    monkeypatch.setattr(O, "make_params", bad)
    with pytest.raises(AssertionError):
        TC.test_per_voxel_strength_driving_force()


def test_strength_ignored_in_driving_force_is_caught(monkeypatch):
    def bad(F, c, prm):  # the phase's mean strength instead of the voxel's own
        s = O.principal_stresses(O.cauchy_undegraded(F, c, prm))
        t = np.maximum(s, 0.0) / prm.sigma_max.mean()
        return np.maximum(np.sum(t * t, axis=0) - 1.0, 0.0)
    monkeypatch.setattr(O, "driving_force", bad)
    with pytest.raises(AssertionError):
        TC.test_per_voxel_strength_driving_force()


def test_history_not_updated_is_caught(monkeypatch):
    from tests import test_oracle_solvers as TSO

    def bad(H_t, F, c, prm):  # the step keeps the last converged history
        return H_t.copy()
    monkeypatch.setattr(O, "history_update", bad)
    with pytest.raises(AssertionError):
        TSO.test_homogeneous_bar_under_stretch_damages_in_closed_form()


def test_staggered_body_skipped_at_equilibrium_is_caught(monkeypatch):
    from tests import test_oracle_solvers as TSO
    good = O.pff_solve
    calls = {"n": 0}

    def bad(H, d0, prm, tol, maxit, stats=None):  # phase field never solved after the first
        calls["n"] += 1
        return d0.copy() if calls["n"] > 1 else good(H, d0, prm, tol, maxit, stats)
    monkeypatch.setattr(O, "pff_solve", bad)
    with pytest.raises(AssertionError):
        TSO.test_homogeneous_bar_under_stretch_damages_in_closed_form()


def test_displacement_without_corner_phase_is_caught(monkeypatch):
    from oracle import fg_oracle_adjoint as A
    from tests import test_oracle_adjoint as TA

    def bad(prm):  # drops exp(-i sum q/2): u placed at the voxel centres, not the corners
        n = O.rotated_frequencies(prm.shape, prm.h)
        nn = np.sum(n * n, axis=0)
        inv = np.divide(1.0, nn, out=np.zeros_like(nn), where=nn > 0.0)
        return -1j * n * inv[None]
    monkeypatch.setattr(A, "displacement_multiplier", bad)
    with pytest.raises(AssertionError):
        TA.test_corner_displacement_inverts_the_corner_stencil((5, 7, 9))


def test_phase_field_without_toughness_division_is_caught(monkeypatch):
    from tests import test_oracle_adjoint as TA

    def bad(H, d0, prm, tol, maxit, stats=None):  # H instead of H g_c / g_c(x)
        Hbar = float(np.mean(H))
        d, it = O.pcg(lambda x: O.pff_apply(x, H, prm), lambda r: O.pff_precond(r, Hbar, prm),
                      2.0 * H, tol, maxit, d0)
        return d
    monkeypatch.setattr(O, "pff_solve", bad)
    with pytest.raises(AssertionError):
        TA.test_damage_does_not_depend_on_the_toughness()


def test_conductivity_with_left_cauchy_green_is_caught(monkeypatch):
    def bad(F_t, c_t, d_t, prm):  # b^{-1} = F^{-T} F^{-1} in place of C^{-1}
        binv = O.tinv(O.tmul(F_t, O.tT(F_t)))
        return prm.D * O.mobility_phi(d_t) * c_t * (1.0 - c_t) * binv
    monkeypatch.setattr(O, "chem_conductivity", bad)
    with pytest.raises(AssertionError):
        TS.test_chem_mode_decay_under_shear_follows_inverse_right_cauchy_green(1, 0)
    with pytest.raises(AssertionError):
        TS.test_chem_step_under_shear_equals_isotropic_step_with_scaled_diffusivity()


def test_conductivity_with_C_not_inverse_is_caught(monkeypatch):
    def bad(F_t, c_t, d_t, prm):  # C in place of C^{-1}
        C = O.tmul(O.tT(F_t), F_t)
        return prm.D * O.mobility_phi(d_t) * c_t * (1.0 - c_t) * C
    monkeypatch.setattr(O, "chem_conductivity", bad)
    with pytest.raises(AssertionError):
        TS.test_chem_mode_decay_under_shear_follows_inverse_right_cauchy_green(1, 0)


def test_mobility_linear_damage_term_is_caught(monkeypatch):
    # 0.1 d in place of 0.1 d^2: phi(0) is unchanged, so only a damaged pin sees it
    monkeypatch.setattr(O, "mobility_phi", lambda d: 0.9 * (1.0 - d) ** 2 + 0.1 * d)
    TS.test_chem_single_mode_decay()  # undamaged pin cannot tell
    with pytest.raises(AssertionError):
        TS.test_chem_mode_decay_with_uniform_damage_follows_mobility(0.25)


def test_crack_energy_length_scale_factor_is_caught(monkeypatch):
    def bad(d, prm, gc_field=None):  # l_c in place of l_c/2 on the gradient term
        xi = O.fd_frequencies(prm.shape, prm.h)
        g = O.irfft3(xi * O.rfft3(d)[None], prm.shape)
        dens = prm.gc * (d * d / (2.0 * prm.lc) + prm.lc * np.sum(g * g, axis=0))
        return float(np.sum(dens) * prm.h[0] * prm.h[1] * prm.h[2])
    monkeypatch.setattr(O, "crack_energy", bad)
    with pytest.raises(AssertionError):
        TS.test_crack_energy_closed_form()


def test_crack_energy_without_voxel_volume_is_caught(monkeypatch):
    good = O.crack_energy
    monkeypatch.setattr(O, "crack_energy",
                        lambda d, prm, gc_field=None: good(d, prm, gc_field) / prm.h[2] * prm.h[0])
    with pytest.raises(AssertionError):
        TS.test_crack_energy_closed_form()


def test_phase_field_with_half_driving_term_is_caught(monkeypatch):
    from tests import test_oracle_solvers as TSO
    good = O.pff_solve

    def bad(H, d0, prm, tol, maxit, stats=None):  # solves A d = H instead of 2H
        return good(0.5 * H, d0, prm, tol, maxit, stats)
    monkeypatch.setattr(O, "pff_solve", bad)
    with pytest.raises(AssertionError):
        TSO.test_coupled_step_output_solves_the_step_equations()


def test_chemistry_with_half_time_step_is_caught(monkeypatch):
    from tests import test_oracle_solvers as TSO
    good = O.chem_solve

    def bad(c_t, F, d_t, dt, *args, **kw):  # the Fick step advanced by dt / 2
        return good(c_t, F, d_t, 0.5 * dt, *args, **kw)
    monkeypatch.setattr(O, "chem_solve", bad)
    with pytest.raises(AssertionError):
        TSO.test_coupled_step_output_solves_the_step_equations()


def test_chemistry_with_final_damage_is_caught(monkeypatch):
    from tests import test_oracle_solvers as TSO
    good = O.chem_solve

    def bad(c_t, F, d_t, dt, *args, **kw):  # the mobility from a damage field not d_t
        return good(c_t, F, np.clip(d_t + 0.5, 0.0, 0.9), dt, *args, **kw)
    monkeypatch.setattr(O, "chem_solve", bad)
    with pytest.raises(AssertionError):
        TSO.test_coupled_step_output_solves_the_step_equations()
