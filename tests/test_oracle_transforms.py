"""Pins for the oracle's transforms and spectral derivatives.

Each check compares the oracle against something other than itself: the DFT
matrix built here from its definition, numpy's FFT (an independent library),
closed-form derivatives of band-limited trigonometric polynomials, and the
paper's Fourier variables of Section 2.3.3.
"""
import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(1234)


def dft_matrix(n, sign):
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n)


@pytest.mark.parametrize("n", list(range(1, 17)) + [24, 32, 48, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1_and_dft1_match_definition(n, sign):
    x = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    ref = dft_matrix(n, sign) @ x
    tol = 1e-13 * max(1.0, np.abs(ref).max()) * max(1, np.log2(max(n, 2)))
    assert np.abs(O.dft1(x, sign) - ref).max() < tol
    assert np.abs(O.fft1(x, sign) - ref).max() < tol


@pytest.mark.parametrize("n", [(8, 4), (16, 32), (1, 8), (64, 64), (6, 10)])
def test_fftn_2d_matches_numpy(n):
    g = O.Grid(n)
    a = RNG.standard_normal(g.shape) + 1j * RNG.standard_normal(g.shape)
    F = O.fftn(g, a, -1)
    assert np.allclose(F, np.fft.fftn(a), rtol=0, atol=1e-12 * np.abs(F).max())
    back = O.fftn(g, F, +1)
    assert np.allclose(back, a, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [(4, 8, 2), (8, 8, 8), (16, 4, 8)])
def test_fftn_3d_matches_numpy_and_parseval(n):
    g = O.Grid(n)
    a = RNG.standard_normal(g.shape)
    F = O.fftn(g, a, -1)
    assert np.allclose(F, np.fft.fftn(a), atol=1e-12 * np.abs(F).max())
    # Parseval: sum |a|^2 = (1/N) sum |F|^2
    assert np.isclose((np.abs(F) ** 2).sum() / a.size, (a ** 2).sum(), rtol=1e-13)


def test_fourier_variables_follow_section_2_3_3():
    # xi(l) = 2 pi l / L for 0 <= l <= N/2, 2 pi (l - N)/L above; Nyquist positive
    N, L = 8, 2.0
    expect = [2 * np.pi * l / L if l <= N // 2 else 2 * np.pi * (l - N) / L for l in range(N)]
    got = [O.xi(l, N, L) for l in range(N)]
    assert np.allclose(got, expect, rtol=1e-15)
    assert O.xi(N // 2, N, L) > 0
    # derivative multiplier: Nyquist zeroed (reading R1), the rest unchanged
    assert O.xi_deriv(N // 2, N, L) == 0.0
    assert all(O.xi_deriv(l, N, L) == O.xi(l, N, L) for l in range(N) if l != N // 2)
    # odd N has no Nyquist index
    assert O.xi_deriv(2, 5, 1.0) == O.xi(2, 5, 1.0) > 0


@pytest.mark.parametrize("n,L", [((16, 8), (1.0, 2.0)), ((32, 32), (1.0, 1.0)),
                                 ((8, 16), (3.0, 0.5))])
def test_gradient_of_trig_polynomial_is_exact(n, L):
    g = O.Grid(n, L)
    nx, ny = n
    Lx, Ly = L
    x = np.arange(nx) * Lx / nx
    y = np.arange(ny) * Ly / ny
    X, Y = np.meshgrid(x, y)  # shape (ny, nx)
    kx, ky = nx // 2 - 1, ny // 2 - 1  # highest non-Nyquist modes
    ax, ay = 2 * np.pi * kx / Lx, 2 * np.pi * ky / Ly
    f = np.sin(ax * X) * np.cos(ay * Y) + 0.3 * np.cos(2 * np.pi * X / Lx + 4 * np.pi * Y / Ly)
    fx = ax * np.cos(ax * X) * np.cos(ay * Y) - 0.3 * 2 * np.pi / Lx * np.sin(
        2 * np.pi * X / Lx + 4 * np.pi * Y / Ly)
    fy = -ay * np.sin(ax * X) * np.sin(ay * Y) - 0.3 * 4 * np.pi / Ly * np.sin(
        2 * np.pi * X / Lx + 4 * np.pi * Y / Ly)
    grad = O.gradient(g, f)
    scale = max(ax, ay)
    assert np.abs(grad[0] - fx).max() < 1e-12 * scale
    assert np.abs(grad[1] - fy).max() < 1e-12 * scale


def test_gradient_3d_trig_polynomial():
    n, L = (8, 16, 4), (1.0, 2.0, 0.5)
    g = O.Grid(n, L)
    z, y, x = np.meshgrid(*(np.arange(n[a]) * L[a] / n[a] for a in (2, 1, 0)), indexing="ij")
    k = [2 * np.pi * 3 / L[0], 2 * np.pi * 2 / L[1], 2 * np.pi * 1 / L[2]]
    f = np.sin(k[0] * x + k[1] * y) * np.cos(k[2] * z)
    grad = O.gradient(g, f)
    assert np.allclose(grad[0], k[0] * np.cos(k[0] * x + k[1] * y) * np.cos(k[2] * z), atol=1e-11)
    assert np.allclose(grad[1], k[1] * np.cos(k[0] * x + k[1] * y) * np.cos(k[2] * z), atol=1e-11)
    assert np.allclose(grad[2], -k[2] * np.sin(k[0] * x + k[1] * y) * np.sin(k[2] * z), atol=1e-11)


def test_nyquist_reading_equals_real_part_of_paper_derivative():
    """R1: zeroing i*xi at the Nyquist index equals Re F^-1[i xi F f] with the
    paper's positive Nyquist xi (what a complex-to-real inverse keeps)."""
    n, L = (16, 8), (1.0, 2.0)
    g = O.Grid(n, L)
    f = RNG.standard_normal(g.shape)
    F = np.fft.fft2(f)
    for a, (na, La) in enumerate(zip(n, L)):
        l = np.arange(na)
        xi = np.where(l <= na // 2, 2 * np.pi * l / La, 2 * np.pi * (l - na) / La)
        mult = 1j * (xi[None, :] if a == 0 else xi[:, None])
        ref = np.fft.ifft2(mult * F)
        assert np.abs(ref.imag).max() > 1e-3  # the paper's form alone is not real
        got = O.gradient(g, f)[a]
        assert np.allclose(got, ref.real, atol=1e-12)


def test_gradient_of_nyquist_mode_vanishes():
    g = O.Grid((8, 8))
    i = np.arange(8)
    f = ((-1.0) ** i)[None, :] * np.ones((8, 1))
    assert np.abs(O.gradient(g, f)).max() < 1e-14
