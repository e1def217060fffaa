"""Pins for Algorithm 1's loop with the stopping rules of Section 2.5
(oracle.run, oracle.delta_m) and for the paper's analytic inputs of Section 3.

Closed forms: with S = 0 the pressure is 0, a uniform m feels neither
activation nor diffusion, and relaxation has exact solutions, so Delta m and
the energy are known along the whole run (gamma = 1: decay by exp(-dt);
gamma = 1/2: |m| decreases by dt per step)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def uniform(g, a, b):
    return np.stack([np.full(g.shape, a), np.full(g.shape, b)])


def test_delta_m_and_energy_closed_form_gamma_one():
    g = O.Grid((16, 8), (1.0, 0.5))
    a, b, dt = 0.7, -0.3, 0.01
    prm = O.Params(c=3.0, D=0.1, gamma=1.0, dt=dt, cg_rtol=1e-12)
    res = O.run(g, prm, np.full(g.shape, 0.2), np.zeros(g.shape), uniform(g, a, b),
                max_steps=6, eps=0.5)
    assert res.reason == 0 and res.steps == 6
    area = 0.5
    for k in range(6):
        assert res.delta_ms[k] == pytest.approx((1 - math.exp(-dt)) / dt, rel=1e-12)
        E = 0.5 * area * (a * a + b * b) * math.exp(-2 * k * dt)  # (1/(2 gamma)) |m|^2 |Omega|
        assert res.energies[k] == pytest.approx(E, rel=1e-12)
    # Delta m is constant: a threshold above it stops after the first step
    res = O.run(g, prm, np.full(g.shape, 0.2), np.zeros(g.shape), uniform(g, a, b),
                max_steps=6, eps=1.0)
    assert res.reason == 1 and res.steps == 1
    assert np.allclose(res.m, uniform(g, a, b) * math.exp(-dt), rtol=1e-14)


def test_delta_m_and_energy_closed_form_gamma_half():
    """gamma = 1/2: |m| <- |m| - dt, so Delta m_k = 1 / (|m0| - k dt) grows and
    E(m^k) = |Omega| (|m0| - k dt) falls linearly."""
    g = O.Grid((8, 8))
    a, b, dt = 0.3, 0.4, 0.02  # |m0| = 0.5
    prm = O.Params(c=1.0, D=0.05, gamma=0.5, dt=dt, cg_rtol=1e-12)
    res = O.run(g, prm, np.full(g.shape, 0.1), np.zeros(g.shape), uniform(g, a, b),
                max_steps=10, eps=1e-3)
    assert res.reason == 0 and res.steps == 10
    for k in range(10):
        nm = 0.5 - k * dt
        assert res.delta_ms[k] == pytest.approx(1.0 / nm, rel=1e-10)
        assert res.energies[k] == pytest.approx(nm, rel=1e-10)


def test_energy_uses_the_pressure_of_the_same_m():
    """energies[k] is E_h(m^k) with the pressure solved from m^k (not from
    m^(k-1)): recompute that pressure independently with PCG."""
    n = 32
    g = O.Grid((n, n))
    w = W.paper_four_sinks(n, 1.5)
    prm = O.Params(c=100.0, D=0.0025, gamma=1.5, dt=0.5, cg_rtol=1e-12, cg_maxit=3000)
    res = O.run(g, prm, w.r, w.S, w.m0, max_steps=3, eps=0, stop_on_energy=False)
    m = w.m0
    b = O.project(g, w.S)
    for k in range(3):
        p, st = O.pcg(g, m, w.r, b, rtol=1e-13, maxit=3000)
        assert res.energies[k] == pytest.approx(O.energy(g, prm, w.r, m, p), rel=1e-9)
        m, _, _ = O.step(g, prm, w.r, w.S, m, p)


def test_energy_rule_stops_after_the_increase_is_seen():
    """The 32^2 four-sinks problem with c = 100, gamma = 1.5, dt = 0.5 lowers
    its energy for eight steps and then raises it (the splitting is not
    unconditionally stable, Remark 2.1)."""
    n = 32
    g = O.Grid((n, n))
    w = W.paper_four_sinks(n, 1.5)
    prm = O.Params(c=100.0, D=0.0025, gamma=1.5, dt=0.5, cg_rtol=1e-12, cg_maxit=3000)
    res = O.run(g, prm, w.r, w.S, w.m0, max_steps=40, eps=0, stop_on_energy=True)
    assert res.reason == 2
    e = res.energies
    assert all(y < x for x, y in zip(e[:-1], e[1:-1]))
    assert e[-1] >= e[-2]
    assert res.energy_step == res.steps - 2 == len(e) - 2
    # without the rule the run continues
    res2 = O.run(g, prm, w.r, w.S, w.m0, max_steps=res.steps + 2, eps=0, stop_on_energy=False)
    assert res2.reason == 0 and res2.steps == res.steps + 2
    assert np.allclose(res2.energies[:len(e)], e, rtol=1e-12)


def test_energy_rule_stops_on_equal_energies():
    """Section 2.5 stops the loop when E_h^k >= E_h^(k-1), equality included.
    With m0 = 0 the conductivity stays 0 (every substep maps 0 to 0) and the
    warm-started pressure repeats exactly, so E_h(m^1) = E_h(m^0) and the loop
    stops after its second body, naming the first."""
    g = O.Grid((16, 16))
    w = W.source_sink_2d(16, steps=1)
    prm = O.Params(c=3.0, D=0.05, gamma=0.75, dt=1e-3, cg_rtol=1e-12)
    res = O.run(g, prm, w.r, w.S, np.zeros((2,) + g.shape), max_steps=10, eps=0.0)
    assert res.reason == 2 and res.steps == 2 and res.energy_step == 0
    assert res.energies[1] == res.energies[0] > 0
    assert not res.m.any()


def test_zero_conductivity_is_a_steady_state_for_the_delta_m_rule():
    """Reading R20: Delta m of a step from m = 0 is 0 (m stays 0), so any
    eps > 0 stops the loop after its first body; with eps = 0 the energy rule
    stops it instead, one body later."""
    g = O.Grid((16, 16))
    w = W.source_sink_2d(16, steps=1)
    prm = O.Params(c=3.0, D=0.05, gamma=0.75, dt=1e-3, cg_rtol=1e-12)
    zero = np.zeros((2,) + g.shape)
    assert O.delta_m(zero, zero, prm.dt) == 0.0
    res = O.run(g, prm, w.r, w.S, zero, max_steps=10, eps=1e-4)
    assert res.reason == 1 and res.steps == 1 and res.delta_ms == [0.0]
    res = O.run(g, prm, w.r, w.S, zero, max_steps=10, eps=0.0)
    assert res.reason == 2 and res.steps == 2


def test_run_stops_on_a_failed_step_and_returns_its_state():
    """Remark 2.1: exp(c^2 |grad p|^2 dt) must stay bounded. When it overflows
    the step reports ENONFINITE, and the loop stops there with reason 3 and
    returns the state that step produced."""
    n = 32
    g = O.Grid((n, n))
    w = W.source_sink_2d(n, steps=1)
    prm = O.Params(c=1e4, D=0.02, gamma=0.5, dt=1e-3, cg_rtol=1e-10)
    m_new, _, st = O.step(g, prm, w.r, w.S, w.m0, np.zeros(g.shape))
    assert st.rc == O.ENONFINITE and not np.isfinite(m_new).all()
    res = O.run(g, prm, w.r, w.S, w.m0, max_steps=5, eps=0.0)
    assert res.reason == 3 and res.steps == 1 and res.energies == []
    assert not np.isfinite(res.m).all()


def test_paper_sources_satisfy_the_solvability_condition():
    """Section 3: int S_4 = 0 and int S_int = 0 (the Gaussians' integral over
    the plane is pi/1000); on a fine grid the node sums agree to quadrature
    accuracy."""
    for n in (256, 512):
        h2 = 1.0 / (n * n)
        assert abs(W.paper_S4(n).sum() * h2) < 1e-12
        assert abs(W.paper_Sint(n).sum() * h2) < 1e-12
    # S_4 is symmetric under x -> 1 - x, y -> 1 - y (node i -> -i mod n) and x <-> y
    S4 = W.paper_S4(64)
    ref = (-np.arange(64)) % 64
    assert np.allclose(S4, S4[:, ref], atol=1e-13) and np.allclose(S4, S4[ref, :], atol=1e-13)
    assert np.allclose(S4, S4.T, atol=1e-15)
    mA, mB, mc = (W.paper_m_ini(64, k) for k in ("A", "B", "const"))
    assert mA.shape == (2, 64, 64) and not mA[1].any() and not mB[1].any()
    assert mA[0, 32, 32] == 1.0 and mB[0, 32, 32] == 1.0 and (mc == 1.0).all()
