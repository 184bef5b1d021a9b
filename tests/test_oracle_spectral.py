"""Pins of the oracle's DFT convention, frequency symbols and projection (Sec. 3.2).

Each check compares the oracle against something other than itself: a brute-force
DFT, real-space finite-difference stencils applied voxel by voxel, or algebraic
properties the projection must have.
"""
import itertools

import numpy as np
import pytest

from oracle import fg_oracle as O

RNG = np.random.default_rng(1234)


def brute_dft3(a):
    nz, ny, nx = a.shape
    out = np.zeros((nz, ny, nx), dtype=complex)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for kz, ky, kx in itertools.product(range(nz), range(ny), range(nx)):
        ph = np.exp(-2j * np.pi * (kz * z / nz + ky * y / ny + kx * x / nx))
        out[kz, ky, kx] = np.sum(a * ph)
    return out


@pytest.mark.parametrize("shape", [(4, 6, 8), (3, 5, 4), (1, 8, 6), (2, 2, 2)])
def test_rfft3_matches_brute_force(shape):
    a = RNG.standard_normal(shape)
    A = O.rfft3(a)
    B = brute_dft3(a)[:, :, : shape[2] // 2 + 1]
    np.testing.assert_allclose(A, B, rtol=0, atol=1e-11)
    np.testing.assert_allclose(O.irfft3(A, shape), a, rtol=0, atol=1e-13)
    # Parseval with the half-spectrum weights
    w = np.full(A.shape[-1], 2.0)
    w[0] = 1.0
    if shape[2] % 2 == 0:
        w[-1] = 1.0
    assert np.isclose(np.sum(w * np.abs(A) ** 2) / a.size, np.sum(a * a), rtol=1e-12)


def shift(u, axis_xyz, s):
    """u(x + s e_axis) for periodic u (..., nz, ny, nx); axis 0 = x, 1 = y, 2 = z."""
    return np.roll(u, -s, axis=-1 - axis_xyz)


def corner_gradient(u, h):
    """Rotated-scheme gradient by its stencil: mean over the 2x2x2 cell of the four
    forward differences along j.  u: (3, nz, ny, nx) -> (3, 3, nz, ny, nx)."""
    out = np.zeros((3, 3) + u.shape[1:])
    for j in range(3):
        others = [m for m in range(3) if m != j]
        acc = np.zeros_like(u)
        for a, b in itertools.product((0, 1), (0, 1)):
            base = shift(shift(u, others[0], a), others[1], b)
            acc += shift(base, j, 1) - base
        out[:, j] = acc / (4.0 * h[j])
    return out


@pytest.mark.parametrize("shape", [(4, 6, 8), (1, 8, 6), (5, 4, 6)])
def test_rotated_symbol_is_corner_stencil(shape):
    h = (0.7, 1.3, 0.9)
    u = RNG.standard_normal((3,) + shape)
    ref = corner_gradient(u, h)
    n = O.rotated_frequencies(shape, h)
    nz, ny, nx = shape
    qx = 2 * np.pi * np.arange(nx // 2 + 1) / nx
    qy = 2 * np.pi * np.fft.fftfreq(ny)
    qz = 2 * np.pi * np.fft.fftfreq(nz)
    phase = np.exp(0.5j * (qx[None, None, :] + qy[None, :, None] + qz[:, None, None]))
    U = O.rfft3(u)
    G = 1j * n[None] * phase[None, None] * U[:, None]
    got = O.irfft3(G, shape)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape", [(4, 6, 8), (1, 8, 6)])
def test_fd_symbols_are_stencils(shape):
    h = (0.7, 1.3, 0.9)
    u = RNG.standard_normal(shape)
    xi = O.fd_frequencies(shape, h)
    U = O.rfft3(u)
    for j in range(3):
        ref = (shift(u, j, 1) - u) / h[j]
        np.testing.assert_allclose(O.irfft3(xi[j] * U, shape), ref, atol=1e-12)
    lap = sum((shift(u, j, 1) - 2 * u + shift(u, j, -1)) / h[j] ** 2 for j in range(3))
    got = O.irfft3(O.fd_laplacian_symbol(shape, h) * U, shape)
    np.testing.assert_allclose(got, -lap, atol=1e-11)


@pytest.mark.parametrize("shape", [(4, 6, 8), (1, 8, 8), (6, 6, 6)])
def test_projection_properties(shape):
    h = (1.0, 1.1, 0.8)
    A = RNG.standard_normal((3, 3) + shape)
    B = RNG.standard_normal((3, 3) + shape)
    GA = O.apply_G(A, h)
    # idempotent
    np.testing.assert_allclose(O.apply_G(GA, h), GA, atol=1e-12)
    # self-adjoint and orthogonal
    assert np.isclose(np.sum(GA * B), np.sum(A * O.apply_G(B, h)), rtol=1e-11)
    assert abs(np.sum((A - GA) * GA)) < 1e-10 * np.sum(A * A)
    # constants are annihilated (zero-mean fluctuation)
    C = np.ones((3, 3) + shape) * RNG.standard_normal((3, 3, 1, 1, 1))
    np.testing.assert_allclose(O.apply_G(C, h), 0.0, atol=1e-13)
    # compatible fields are reproduced (rotated-scheme gradients of periodic u)
    u = RNG.standard_normal((3,) + shape)
    g = corner_gradient(u, h)
    np.testing.assert_allclose(O.apply_G(g, h), g, atol=1e-11)
    # output is curl free in the scheme: n_k A'_ij = n_j A'_ik
    n = O.rotated_frequencies(shape, h)
    Ah = O.project_G(O.rfft3(A), n)
    for i, j, k in itertools.product(range(3), repeat=3):
        np.testing.assert_allclose(n[k] * Ah[i, j], n[j] * Ah[i, k], atol=1e-9)


def test_null_modes_are_zero():
    shape = (4, 4, 4)
    n = O.rotated_frequencies(shape, (1.0, 1.0, 1.0))
    n2 = np.sum(n * n, axis=0)
    # two axes at Nyquist: every component vanishes exactly
    assert n2[2, 2, 0] == 0.0 and n2[0, 2, 2] == 0.0 and n2[2, 0, 2] == 0.0
    assert n2[0, 0, 0] == 0.0
    # mean, plus every (kz, ky, kx) with at least two indices at Nyquist:
    # kx=ky=2 (4 kz) + kx=kz=2 (4 ky) + ky=kz=2 (3 kx) - 2 repeats of (2,2,2)
    assert np.count_nonzero(n2 == 0.0) == 1 + 4 + 4 + 3 - 2
