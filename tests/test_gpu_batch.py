"""Batched parameter sweep: one CUDA graph launch advances several contexts
of mixed grids, parameters and precisions.  Each instance must reproduce its
solo run bit for bit (same kernels, same launch shapes, independent chains),
and the instances follow the FP64 oracle."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import hc, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu


def solver_for(hc, w, precision="fp32_refined"):
    s = hc.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision=precision,
                  cg_rtol=w.cg_rtol, cg_maxit=2000)
    s.set_r(w.r)
    s.set_source(w.S)
    s.set_m(w.m0)
    return s


def test_batch_matches_solo_runs_bitwise(hc):
    cases = [(0, "fp32_refined"), (1, "fp32_refined"), (2, "fp32_refined_df"), (13, "fp64"),
             (29, "fp32_refined")]
    ws = [W.sweep_instance(i) for i, _ in cases]
    solo = []
    for w, (i, prec) in zip(ws, cases):
        with solver_for(hc, w, prec) as s:
            st = s.step(3)
            solo.append((s.get_m(), s.get_p(), st.cg_iters))
    solvers = [solver_for(hc, w, prec) for w, (i, prec) in zip(ws, cases)]
    with hc.Batch(solvers) as b:
        stats = b.step(3)
    for s, st, (m, p, it) in zip(solvers, stats, solo):
        assert st.status == 0
        assert np.array_equal(s.get_m(), m)
        assert np.array_equal(s.get_p(), p)
        assert st.cg_iters == it
        s.close()


def test_batch_instance_follows_oracle(hc):
    w = W.sweep_instance(3)  # 128^2, c=5, D=0.02, gamma=0.5
    g = O.Grid(w.n, w.L)
    prm = O.Params(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-10, cg_maxit=2000)
    m, p = w.m0.copy(), np.zeros(g.shape)
    for _ in range(4):
        m, p, _ = O.step(g, prm, w.r, w.S, m, p)
    other = W.sweep_instance(7)
    s1, s2 = solver_for(hc, w), solver_for(hc, other)
    with hc.Batch([s1, s2]) as b:
        for _ in range(2):
            stats = b.step(2)
            assert all(x.rel_residual <= w.cg_rtol for x in stats)
    assert rel_l2(s1.get_m(), m) <= 1e-5
    s1.close()
    s2.close()


def test_batch_arguments(hc):
    from paper_2606_06720_gb300 import _binding as Bd
    w = W.sweep_instance(0)
    with solver_for(hc, w) as s:
        arr = (C.c_void_p * 2)(s.ctx.value, s.ctx.value)
        b = C.c_void_p()
        assert Bd.hc_batch_create(C.byref(b), arr, 2, None) == hc.HC_EINVAL
        assert Bd.hc_batch_create(C.byref(b), arr, 0, None) == hc.HC_EINVAL
        assert Bd.hc_batch_step(None, 1, None) == hc.HC_EINVAL
