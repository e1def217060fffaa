"""The mixed-radix FP64 path: 2D grids whose sizes are not powers of two
(N = 2^a 3^b 5^c), among them the paper's N = 50 2^k convergence grids
(Section 4).  Against the oracle, whose transforms are direct DFTs on such
sizes: the transform, the spectral gradient, the pressure operator, steps
(FP64 bound 1e-10 per step), the diagnostics energy, and Algorithm 1's loop."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import hc, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu

# even, odd and mixed sizes: 50 = 2 5^2, 100, 200, 45 = 3^2 5, 75 = 3 5^2, 12 = 4 3, 4
SIZES = [(50, 50), (100, 100), (200, 200), (45, 75), (12, 20), (4, 6), (30, 64)]


def solver(hc, n, L=(1.0, 1.0), **kw):
    args = dict(c=10.0, D=0.05, gamma=0.75, dt=1e-3, precision="fp64", cg_rtol=1e-12,
                cg_maxit=5000)
    args.update(kw)
    return hc.Solver(n, L, **args)


def fields(n, seed, L=(1.0, 1.0)):
    rng = np.random.default_rng(seed)
    shape = (n[1], n[0])
    m = rng.uniform(0.0, 0.6, (2,) + shape)
    r = rng.uniform(0.05, 0.2, shape)
    S = W.minus_mean(W.gaussian(n, (0.3 * L[0], 0.5 * L[1]), 0.12, L)
                     - W.gaussian(n, (0.7 * L[0], 0.4 * L[1]), 0.12, L))
    return m, r, S


@pytest.mark.parametrize("n", SIZES)
def test_spectrum_matches_the_oracle_dft(hc, n):
    g = O.Grid(n)
    f = np.random.default_rng(1).standard_normal(g.shape)
    with solver(hc, n) as s:
        assert s.generic
        got = s.spectrum(f)
    want = O.fftn(g, f)[:, : n[0] // 2 + 1]
    assert got.shape == want.shape
    assert rel_l2(got, want) < 1e-13


@pytest.mark.parametrize("n", SIZES)
def test_gradient_and_operator_match_the_oracle(hc, n):
    L = (1.0, 0.7)
    g = O.Grid(n, L)
    m, r, S = fields(n, 2, L)
    p = np.random.default_rng(3).standard_normal(g.shape)
    f = np.random.default_rng(4).standard_normal(g.shape)
    with solver(hc, n, L) as s:
        s.set_r(r)
        s.set_m(m)
        s.set_p(p)
        grad = s.gradient()
        Af = s.apply_operator(f)
    assert rel_l2(grad, O.gradient(g, O.project(g, p))) < 1e-12
    assert rel_l2(Af, O.apply_A(g, m, r, O.project(g, f))) < 1e-12


@pytest.mark.parametrize("n", [(50, 50), (100, 100), (45, 75), (12, 20)])
@pytest.mark.parametrize("use_graph", [True, False])
def test_steps_match_the_oracle(hc, n, use_graph):
    """Four FP64 steps, each within 1e-10 of the oracle's (relative L2 of m
    and p), with CG iteration counts within one."""
    g = O.Grid(n)
    m, r, S = fields(n, 5)
    prm = O.Params(c=10.0, D=0.05, gamma=0.75, dt=1e-3, cg_rtol=1e-12, cg_maxit=5000)
    mo, po = m.copy(), np.zeros(g.shape)
    with solver(hc, n, use_graph=use_graph) as s:
        s.set_r(r)
        s.set_source(S)
        s.set_m(m)
        for _ in range(4):
            st = s.step(1)
            mo, po, sto = O.step(g, prm, r, S, mo, po)
            assert st.status == 0 and st.rel_residual <= 1e-12
            assert abs(st.cg_iters - sto.cg_iters) <= 1
            assert rel_l2(s.get_m(), mo) < 1e-10
            assert rel_l2(s.get_p(), po) < 1e-10


@pytest.mark.parametrize("n", [50, 100])
def test_paper_convergence_setup_against_the_oracle(hc, n):
    """Section 4's convergence setup (S_int, m^A, c = 100, gamma = 0.75,
    D = 0.01, dt = 0.05) at N = 50 and 100: ten steps with the Kbar
    preconditioner, within 1e-10 of the oracle per step."""
    w = W.paper_convergence(n, steps=10)
    g = O.Grid(w.n, w.L)
    prm = O.Params(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-11, cg_maxit=5000, precond=1)
    mo, po = w.m0.copy(), np.zeros(g.shape)
    with hc.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision="fp64",
                   cg_rtol=1e-11, cg_maxit=5000, precond="kbar") as s:
        s.set_r(w.r)
        s.set_source(w.S)
        s.set_m(w.m0)
        for k in range(10):
            st = s.step(1)
            mo, po, _ = O.step(g, prm, w.r, w.S, mo, po)
            assert st.status == 0
            assert rel_l2(s.get_m(), mo) < 1e-10, k
            assert rel_l2(s.get_p(), po) < 1e-10, k


def test_energy_and_run_loop_match_the_oracle(hc):
    """Diagnostics of Section 2.5 and Algorithm 1's loop on a 60 x 45 grid:
    the energy and Delta m of each step within 1e-10, and hc_run stops on the
    Delta m rule at the oracle's step with the oracle's state."""
    n = (60, 45)
    g = O.Grid(n)
    m, r, S = fields(n, 7)
    prm = O.Params(c=10.0, D=0.05, gamma=0.75, dt=1e-3, cg_rtol=1e-12, cg_maxit=5000)
    ref = O.run(g, prm, r, S, m, max_steps=6, eps=0, stop_on_energy=False)
    with solver(hc, n, diagnostics=True) as s:
        s.set_r(r)
        s.set_source(S)
        s.set_m(m)
        for k in range(6):
            st = s.step(1)
            assert st.energy_valid == 1
            assert st.energy == pytest.approx(ref.energies[k], rel=1e-10), k
            assert st.delta_m == pytest.approx(ref.delta_ms[k], rel=1e-9), k
    dm = np.array(O.run(g, prm, r, S, m, max_steps=30, eps=0, stop_on_energy=False).delta_ms)
    eps = 0.5 * (dm[12] + dm[13])
    ref = O.run(g, prm, r, S, m, max_steps=30, eps=eps, stop_on_energy=True)
    assert ref.reason == 1
    with solver(hc, n) as s:
        s.set_r(r)
        s.set_source(S)
        s.set_m(m)
        st = s.run(30, eps=eps)
        assert st.stop_reason == hc.HC_STOP_DELTA_M and st.steps == ref.steps
        assert rel_l2(s.get_m(), ref.m) < 1e-10


def test_unsupported_on_generic_grids(hc):
    """A mixed-radix grid takes FP64 plain only; the adjoint, tuning and kernel
    timing are not offered there."""
    from paper_2606_06720_gb300 import HuCaiError
    with pytest.raises(HuCaiError):
        hc.Solver((50, 50), (1.0, 1.0), c=1.0, D=0.1, gamma=1.0, dt=1e-3, precision="fp32_refined")
    with solver(hc, (50, 50)) as s:
        with pytest.raises(HuCaiError):
            s.time_kernel("cg_apply")
