"""Pins for the oracle's whole step (Algorithm 1 loop body) and its energy
(Section 2.5, eq. energy): the energy identity of the pressure equation,
energy dissipation for small dt (the L2 gradient-flow structure of Section
1.1), reflection symmetry, and closed-form special cases of the splitting.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

RNG = np.random.default_rng(5)


def smooth_problem(n=32):
    g = O.Grid((n, n))
    X, Y = np.meshgrid(np.arange(n) / n, np.arange(n) / n)
    m = np.stack([0.5 + 0.2 * np.cos(2 * np.pi * Y), 0.4 + 0.1 * np.sin(2 * np.pi * X)])
    r = np.full(g.shape, 0.1)
    S = W.minus_mean(W.gaussian((n, n), (0.3, 0.5), 0.08) - W.gaussian((n, n), (0.7, 0.5), 0.08))
    return g, m, r, S


def test_energy_identity_of_the_pressure_equation():
    """For p solving A p = S: sum (m.grad p)^2 + r |grad p|^2 = sum p S (discrete
    integration by parts with the symmetric spectral derivative)."""
    g, m, r, S = smooth_problem()
    b = O.project(g, S)
    p, st = O.pcg(g, m, r, b, rtol=1e-13)
    gp = O.gradient(g, p)
    lhs = (((m * gp).sum(0)) ** 2 + r * (gp ** 2).sum(0)).sum()
    rhs = (p * b).sum()
    assert np.isclose(lhs, rhs, rtol=1e-10)
    # so with D = 0 and gamma = 1: E = (c^2/2) h sum p S + (1/2) h sum |m|^2
    prm = O.Params(c=3.0, D=0.0, gamma=1.0, dt=1e-3)
    h = 1.0 / g.npts
    E = O.energy(g, prm, r, m, p)
    assert np.isclose(E, h * (0.5 * 9.0 * rhs + 0.5 * (m ** 2).sum()), rtol=1e-10)


def test_energy_non_increasing_for_small_dt():
    g, m, r, S = smooth_problem()
    prm = O.Params(c=5.0, D=0.05, gamma=0.75, dt=2e-4, cg_rtol=1e-12)
    p = np.zeros(g.shape)
    energies = []
    for _ in range(6):
        m_new, p, st = O.step(g, prm, r, S, m, p)  # p solves for the current m
        assert st.rc == O.OK
        energies.append(O.energy(g, prm, r, m, p))
        m = m_new
    assert all(b < a for a, b in zip(energies, energies[1:]))


def test_step_preserves_diagonal_reflection_symmetry():
    n = 32
    g = O.Grid((n, n))
    S = W.minus_mean(W.gaussian((n, n), (0.3, 0.3), 0.06) - W.gaussian((n, n), (0.7, 0.7), 0.06))
    S = 0.5 * (S + S.T)
    U = RNG.uniform(0, 1, (n, n))
    m = np.stack([U, U.T])  # m_x(x, y) = m_y(y, x)
    r = np.full(g.shape, 0.1)
    prm = O.Params(c=10.0, D=0.05, gamma=0.75, dt=1e-3, cg_rtol=1e-12)
    p = np.zeros(g.shape)
    for _ in range(3):
        m, p, st = O.step(g, prm, r, S, m, p)
    assert np.allclose(p, p.T, atol=1e-10)
    assert np.allclose(m[0], m[1].T, atol=1e-10)


def test_step_special_case_pure_relaxation():
    """c = 0 and D = 0, gamma = 1: activation and diffusion are identities and
    m^{k+1} = m^k exp(-dt) exactly (eq. m_relaxation_discrete)."""
    g = O.Grid((16, 8), (1.0, 2.0))
    m = RNG.uniform(0, 1, (2,) + g.shape)
    r = np.full(g.shape, 0.1)
    S = O.project(g, RNG.standard_normal(g.shape))
    prm = O.Params(c=0.0, D=0.0, gamma=1.0, dt=0.01)
    m2, p2, st = O.step(g, prm, r, S, m, np.zeros(g.shape))
    assert np.allclose(m2, m * np.exp(-0.01), rtol=1e-13)
    # p is the solution for the incoming m
    assert np.abs(O.apply_A(g, m, r, p2) - S).max() < 1e-8 * np.abs(S).max()


def test_step_special_case_relaxation_commutes_with_diffusion():
    """c = 0, gamma = 1: m^{k+1} = exp(-dt) * heat(m^k) for a single Fourier mode."""
    n, L = (16, 16), (1.0, 1.0)
    g = O.Grid(n, L)
    X, Y = np.meshgrid(np.arange(16) / 16, np.arange(16) / 16)
    mode = np.cos(2 * np.pi * (2 * X + 3 * Y))
    m = np.stack([mode, -mode])
    D, dt = 0.1, 0.01
    prm = O.Params(c=0.0, D=D, gamma=1.0, dt=dt)
    S = O.project(g, RNG.standard_normal(g.shape))
    m2, _, _ = O.step(g, prm, np.full(g.shape, 0.1), S, m, np.zeros(g.shape))
    lam = (2 * np.pi) ** 2 * 13
    assert np.allclose(m2, m * np.exp(-dt) * np.exp(-D * D * lam * dt), atol=1e-13)


def test_step_follows_algorithm_1_order():
    """Algorithm 1: solve p^{k+1} with m^k (warm start p^k), then activation
    with grad p^{k+1}, relaxation, diffusion (R6, R11)."""
    g = O.Grid((16, 32), (1.0, 2.0))
    m = RNG.uniform(0, 1, (2,) + g.shape)
    r = W.smooth_r((16, 32), 3, (1.0, 2.0))
    S = RNG.standard_normal(g.shape)
    prm = O.Params(c=4.0, D=0.1, gamma=0.75, dt=1e-3, cg_rtol=1e-12)
    p0 = RNG.standard_normal(g.shape)
    m2, p2, st = O.step(g, prm, r, S, m, p0)
    p_ref, _ = O.pcg(g, m, r, O.project(g, S), x0=p0, rtol=1e-12)
    assert np.array_equal(p2, p_ref)
    a = O.activation(m, O.gradient(g, p_ref), prm.c, prm.dt)
    b = O.relaxation(a, prm.gamma, prm.dt)
    c = O.diffusion(g, b, prm.D, prm.dt)
    assert np.array_equal(m2, c)


def test_step_3d_runs_and_is_symmetric_in_swapped_axes():
    n = 8
    g = O.Grid((n, n, n))
    S = W.minus_mean(W.gaussian((n, n, n), (0.3, 0.5, 0.5), 0.1) - W.gaussian((n, n, n), (0.7, 0.5, 0.5), 0.1))
    # S symmetric under y <-> z (numpy axes 0 <-> 1); m_y and m_z swap with it
    U = RNG.uniform(0, 0.5, (n, n, n))
    V = RNG.uniform(0, 0.5, (n, n, n))
    V = 0.5 * (V + V.transpose(1, 0, 2))
    m = np.stack([V, U, U.transpose(1, 0, 2)])
    prm = O.Params(c=5.0, D=0.05, gamma=0.75, dt=1e-3, cg_rtol=1e-12)
    r = np.full(g.shape, 0.1)
    m2, p2, st = O.step(g, prm, r, S, m, np.zeros(g.shape))
    assert st.rc == O.OK
    assert np.allclose(p2, p2.transpose(1, 0, 2), atol=1e-11)
    assert np.allclose(m2[1], m2[2].transpose(1, 0, 2), atol=1e-11)
    assert np.allclose(m2[0], m2[0].transpose(1, 0, 2), atol=1e-11)


def test_step_reports_nonconvergence_but_advances():
    g, m, r, S = smooth_problem(16)
    prm = O.Params(c=5.0, D=0.05, gamma=0.75, dt=1e-3, cg_rtol=1e-14, cg_maxit=2)
    m2, p2, st = O.step(g, prm, r, S, m, np.zeros(g.shape))
    assert st.rc == O.ENOCONV and st.cg_iters == 2
    assert not np.array_equal(m2, m)


def test_results_do_not_depend_on_the_thread_count():
    """The oracle's parallel loops write disjoint entries and its sums run in a
    fixed order, so a step gives bit-identical results on 1 and on 8 threads."""
    import workloads as W
    w = W.source_sink_2d(32, steps=1)
    g = O.Grid(w.n, w.L)
    prm = O.Params(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-10)
    before = O.get_threads()
    try:
        outs = []
        for t in (1, 8):
            O.set_threads(t)
            outs.append(O.step(g, prm, w.r, w.S, w.m0, np.zeros(g.shape)))
    finally:
        O.set_threads(before)
    (m1, p1, s1), (m8, p8, s8) = outs
    assert np.array_equal(m1, m8) and np.array_equal(p1, p8) and s1.cg_iters == s8.cg_iters
