"""Pins for the oracle's splitting substeps (Section 2.3).

Activation: the matrix exponential of c^2 dt g g^T (scipy's expm, a textbook
special case) and brute-force RK4 of dm/dt = c^2 (m.g) g.  Relaxation: the
closed forms for gamma = 1 and gamma = 1/2 and brute-force RK4 of the radial
ODE for other gamma.  Diffusion: exact decay of single Fourier modes.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle as O

RNG = np.random.default_rng(7)


def rk4(f, y, T, nsteps):
    h = T / nsteps
    for _ in range(nsteps):
        k1 = f(y); k2 = f(y + 0.5 * h * k1); k3 = f(y + 0.5 * h * k2); k4 = f(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return y


@pytest.mark.parametrize("dim", [2, 3])
def test_activation_matches_matrix_exponential(dim):
    npts = 40
    m = RNG.standard_normal((dim, npts))
    g = RNG.standard_normal((dim, npts))
    c, dt = 3.0, 0.05
    out = O.activation(m, g, c, dt)
    for q in range(npts):
        ref = expm(c * c * dt * np.outer(g[:, q], g[:, q])) @ m[:, q]
        assert np.allclose(out[:, q], ref, rtol=1e-12, atol=1e-12)


def test_activation_matches_rk4_and_zero_gradient():
    m = np.array([[0.3, 1.0, 0.0], [0.7, -0.2, 0.5]])
    g = np.array([[0.4, 0.0, 0.0], [-0.9, 0.0, 0.0]])  # second and third points: g = 0
    c, dt = 2.0, 0.1
    out = O.activation(m, g, c, dt)
    gg = g[:, 0]
    ref = rk4(lambda v: c * c * (v @ gg) * gg, m[:, 0], dt, 4000)
    assert np.allclose(out[:, 0], ref, rtol=1e-11)
    assert np.array_equal(out[:, 1:], m[:, 1:])  # |grad p| = 0: unchanged


def test_relaxation_gamma_one_and_one_half_closed_forms():
    m = RNG.standard_normal((2, 30))
    dt = 0.07
    assert np.allclose(O.relaxation(m, 1.0, dt), m * np.exp(-dt), rtol=1e-15)
    out = O.relaxation(m, 0.5, dt)
    nm = np.sqrt((m ** 2).sum(0))
    ref = m * np.maximum(nm - dt, 0.0) / nm
    assert np.allclose(out, ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("gamma", [0.75, 0.8, 0.9, 1.5, 2.0])
def test_relaxation_matches_radial_rk4(gamma):
    # |m| well above extinction so the radial ODE d|m|/dt = -|m|^{2 gamma - 1} is smooth
    m = RNG.uniform(0.5, 1.5, (3, 10)) * RNG.choice([-1, 1], (3, 10))
    dt = 0.05
    out = O.relaxation(m, gamma, dt)
    for q in range(m.shape[1]):
        r0 = np.linalg.norm(m[:, q])
        rT = rk4(lambda s: -s ** (2 * gamma - 1), r0, dt, 2000)
        assert np.allclose(out[:, q], m[:, q] / r0 * rT, rtol=1e-11)


def test_relaxation_extinction_and_zero():
    gamma, dt = 0.75, 0.1
    # extinction time |m0|^{2(1-gamma)} / (2(1-gamma)): below dt -> clipped to 0
    small = 0.001
    assert small ** (2 * (1 - gamma)) / (2 * (1 - gamma)) < dt
    m = np.array([[small, 0.0, 0.3], [0.0, 0.0, 0.4]])
    out = O.relaxation(m, gamma, dt)
    assert np.all(out[:, 0] == 0)
    assert np.all(out[:, 1] == 0)  # |m| = 0 stays 0
    assert np.all(out[:, 2] != 0)


@pytest.mark.parametrize("n,L", [((16, 8), (1.0, 2.0)), ((8, 32), (0.5, 1.0))])
def test_diffusion_single_mode_decay(n, L):
    g = O.Grid(n, L)
    D, dt = 0.3, 0.01
    X, Y = np.meshgrid(np.arange(n[0]) * L[0] / n[0], np.arange(n[1]) * L[1] / n[1])
    k, l = 3, 2
    mode = np.cos(2 * np.pi * (k * X / L[0] + l * Y / L[1]))
    m = np.stack([mode, 2.0 * mode])
    lam = (2 * np.pi) ** 2 * ((k / L[0]) ** 2 + (l / L[1]) ** 2)
    out = O.diffusion(g, m, D, dt)
    assert np.allclose(out, m * np.exp(-D * D * lam * dt), atol=1e-13)
    # Nyquist mode along x keeps the positive Nyquist wavenumber pi N / L (squared)
    nyq = ((-1.0) ** np.arange(n[0]))[None, :] * np.ones((n[1], 1))
    out = O.diffusion(g, np.stack([nyq, 0 * nyq]), D, dt)
    decay = np.exp(-D * D * (np.pi * n[0] / L[0]) ** 2 * dt)
    assert np.allclose(out[0], decay * nyq, atol=1e-13)


def test_diffusion_3d_mode():
    n, L = (8, 4, 16), (1.0, 0.5, 2.0)
    g = O.Grid(n, L)
    z, y, x = np.meshgrid(*(np.arange(n[a]) * L[a] / n[a] for a in (2, 1, 0)), indexing="ij")
    mode = np.sin(2 * np.pi * (2 * x / L[0] + 1 * y / L[1] + 3 * z / L[2]))
    lam = (2 * np.pi) ** 2 * ((2 / L[0]) ** 2 + (1 / L[1]) ** 2 + (3 / L[2]) ** 2)
    D, dt = 0.1, 0.02
    out = O.diffusion(g, np.stack([mode, mode, -mode]), D, dt)
    assert np.allclose(out[2], -mode * np.exp(-D * D * lam * dt), atol=1e-13)
