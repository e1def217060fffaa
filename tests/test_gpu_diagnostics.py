"""GPU diagnostics of Section 2.5 (energy E_h and Delta m) and Algorithm 1's
loop with its stopping rules (hc_run) against the oracle (oracle.run), in 2D
and 3D, both precisions, graph and host-loop modes."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import hc, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu

TOL_E = {"fp64": 1e-10, "fp32_refined": 2e-5}


def solver(hc, w, precision, **kw):
    args = dict(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision=precision, cg_rtol=1e-12,
                cg_maxit=5000, diagnostics=True)
    args.update(kw)
    s = hc.Solver(w.n, w.L, **args)
    s.set_r(w.r)
    s.set_source(w.S)
    s.set_m(w.m0)
    return s


def oracle_prm(w, **kw):
    args = dict(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-12, cg_maxit=5000)
    args.update(kw)
    return O.Params(**args)


def problem_2d(n=64):
    w = W.source_sink_2d(n, steps=10, gamma=0.75)
    w.c, w.dt = 10.0, 1e-3
    return w


def problem_3d(n=16):
    w = W.source_sink_3d(n)
    w.c, w.dt = 5.0, 1e-3
    return w


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
@pytest.mark.parametrize("dim", [2, 3])
def test_energy_and_delta_m_per_step_match_oracle(hc, precision, dim):
    w = problem_2d() if dim == 2 else problem_3d()
    g = O.Grid(w.n, w.L)
    # the refined path holds m and r in FP32: give the oracle the same inputs
    cast = (lambda a: a) if precision == "fp64" else (lambda a: a.astype(np.float32).astype(np.float64))
    ref = O.run(g, oracle_prm(w), cast(w.r), w.S, cast(w.m0), max_steps=5, eps=0,
                stop_on_energy=False)
    with solver(hc, w, precision) as s:
        for k in range(5):
            st = s.step(1)
            assert st.energy_valid == 1
            assert st.energy == pytest.approx(ref.energies[k], rel=TOL_E[precision]), k
            assert st.delta_m == pytest.approx(ref.delta_ms[k], rel=TOL_E[precision] * 10), k


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_gamma0_energy_is_the_log_term_like_the_oracle(hc, precision):
    """Reading R21: at gamma = 0 the energy's relaxation term is h sum ln|m|.
    With |m| kept away from 0 it is finite and matches the oracle step by step;
    once the relaxation extinguishes points (|m|^2 < 2 dt) and diffusion leaves
    a zero, it is -inf, and the energy rule stops the loop at the oracle's step."""
    w = problem_2d()
    w.gamma = 0.0
    w.m0 = w.m0 + 0.5
    g = O.Grid(w.n, w.L)
    cast = (lambda a: a) if precision == "fp64" else (lambda a: a.astype(np.float32).astype(np.float64))
    ref = O.run(g, oracle_prm(w), cast(w.r), w.S, cast(w.m0), max_steps=5, eps=0,
                stop_on_energy=False)
    assert all(np.isfinite(ref.energies))
    with solver(hc, w, precision) as s:
        for k in range(5):
            st = s.step(1)
            assert st.energy_valid == 1
            assert st.energy == pytest.approx(ref.energies[k], rel=TOL_E[precision]), k
    w = W.source_sink_2d(32, steps=10, gamma=0.0)
    w.c, w.dt = 10.0, 0.05
    g = O.Grid(w.n, w.L)
    ref = O.run(g, oracle_prm(w), cast(w.r), w.S, cast(w.m0), max_steps=10, eps=0,
                stop_on_energy=True)
    assert ref.reason == 2 and np.isneginf(ref.energies[-1]) and np.isfinite(ref.energies[0])
    with solver(hc, w, precision) as s:
        st = s.run(10, eps=0, stop_on_energy=True)
        assert st.stop_reason == hc.HC_STOP_ENERGY
        assert st.steps == ref.steps and st.energy_step == ref.energy_step
        assert np.isneginf(st.energy)


def test_energy_validity_follows_the_diagnostics_switch(hc):
    """The energy of a state needs its gradient norm, computed by hc_set_m or
    by a step that ran with diagnostics on."""
    w = problem_2d(32)
    with solver(hc, w, "fp64", diagnostics=False) as s:
        st = s.step(2)
        assert st.energy_valid == 0 and st.delta_m == 0.0
        s.set_params(diagnostics=True)
        st = s.step(1)  # its starting m came from a step without diagnostics
        assert st.energy_valid == 0 and st.delta_m > 0
        st = s.step(1)
        assert st.energy_valid == 1
        s.set_m(w.m0)   # set_m makes the gradient norm of the new m
        st = s.step(1)
        assert st.energy_valid == 1


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_run_stops_on_delta_m_like_the_oracle(hc, precision, use_graph):
    w = problem_2d(64)
    g = O.Grid(w.n, w.L)
    ref = O.run(g, oracle_prm(w), w.r, w.S, w.m0, max_steps=40, eps=0, stop_on_energy=False)
    dm = np.array(ref.delta_ms)
    # a threshold half-way between two consecutive values, where they differ most
    k = 8 + int(np.argmax(np.abs(np.diff(dm[8:30]))))
    eps = 0.5 * (dm[k] + dm[k + 1])
    assert abs(dm[k] - dm[k + 1]) > 1e-3 * dm[k]
    k_stop = next(i for i in range(len(dm)) if dm[i] <= eps)
    assert all(abs(dm[i] - eps) > 1e-4 * eps for i in range(k_stop + 1))  # no near-ties
    ref = O.run(g, oracle_prm(w), w.r, w.S, w.m0, max_steps=40, eps=eps, stop_on_energy=True)
    assert ref.reason == 1 and ref.steps == k_stop + 1
    with solver(hc, w, precision, use_graph=use_graph) as s:
        st = s.run(40, eps=eps, stop_on_energy=True)
        assert st.stop_reason == hc.HC_STOP_DELTA_M
        assert st.steps == ref.steps
        assert st.delta_m <= eps
        tol = 1e-10 if precision == "fp64" else 1e-5
        assert rel_l2(s.get_m(), ref.m) < tol
        # back to plain stepping: no stop reason
        assert s.step(1).stop_reason == hc.HC_STOP_NONE


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_run_stops_on_energy_increase_like_the_oracle(hc, precision, use_graph):
    """The 32^2 four-sinks case (c = 100, gamma = 1.5, dt = 0.5): the energy
    falls for eight steps, then rises by ~6%; the loop stops after the step
    that sees the increase."""
    w = W.paper_four_sinks(32, 1.5)
    w.c, w.dt = 100.0, 0.5
    g = O.Grid(w.n, w.L)
    ref = O.run(g, oracle_prm(w), w.r, w.S, w.m0, max_steps=40, eps=1e-4, stop_on_energy=True)
    assert ref.reason == 2
    with solver(hc, w, precision, use_graph=use_graph, diagnostics=False) as s:
        st = s.run(40, eps=1e-4, stop_on_energy=True)
        assert st.stop_reason == hc.HC_STOP_ENERGY
        assert st.steps == ref.steps and st.energy_step == ref.energy_step
        assert st.energy == pytest.approx(ref.energies[-1], rel=TOL_E[precision] * 100)
        if precision == "fp64":
            assert rel_l2(s.get_m(), ref.m) < 1e-9
        # hc_run forced the diagnostics on for the call only
        assert s.step(1).energy_valid == 0


def test_run_limits_and_graph_gate(hc):
    """max_steps reached (no rule fires), eps <= 0 disables the Delta m rule,
    a gated graph skips steps after a stop, and hc_run with 0 steps is a no-op."""
    w = problem_2d(32)
    with solver(hc, w, "fp32_refined") as s:
        st = s.run(7, eps=0, stop_on_energy=False)
        assert st.stop_reason == hc.HC_STOP_NONE and st.steps == 7
        m7 = s.get_m()
        st = s.run(0)
        assert st.steps == 0
        assert np.array_equal(s.get_m(), m7)
    # a huge eps stops after one step although 37 launches are allowed (the
    # first chunk launches 16 gated steps; 15 of them must skip on the GPU)
    with solver(hc, w, "fp32_refined") as s:
        st = s.run(37, eps=1e9)
        assert st.stop_reason == hc.HC_STOP_DELTA_M and st.steps == 1
        m1 = s.get_m()
    with solver(hc, w, "fp32_refined") as s:
        s.step(1)
        assert np.array_equal(s.get_m(), m1)


def test_run_3d_delta_m_stop(hc):
    w = problem_3d(16)
    g = O.Grid(w.n, w.L)
    ref = O.run(g, oracle_prm(w), w.r, w.S, w.m0, max_steps=30, eps=0, stop_on_energy=False)
    dm = np.array(ref.delta_ms)
    k = 5 + int(np.argmax(np.abs(np.diff(dm[5:25]))))
    eps = 0.5 * (dm[k] + dm[k + 1])
    k_stop = next(i for i in range(len(dm)) if dm[i] <= eps)
    assert all(abs(dm[i] - eps) > 1e-6 * eps for i in range(k_stop + 1))
    ref = O.run(g, oracle_prm(w), w.r, w.S, w.m0, max_steps=30, eps=eps, stop_on_energy=True)
    assert ref.reason == 1
    with solver(hc, w, "fp64") as s:
        st = s.run(30, eps=eps)
        assert st.stop_reason == hc.HC_STOP_DELTA_M and st.steps == ref.steps
        assert rel_l2(s.get_m(), ref.m) < 1e-10
        assert st.energy == pytest.approx(ref.energies[-1], rel=1e-10)
