"""Batched parameter sweep: one CUDA graph launch advances several contexts
of mixed grids, parameters and precisions.  2D refined contexts of one grid
size form a size class whose passes are batched launches over all members;
the others run chains of their own.  Each instance must reproduce its solo
run bit for bit (the same kernel bodies and launch shapes, its own loops),
and every member follows the FP64 oracle at its precision's tolerance."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import hc, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu


def solver_for(hc, w, precision="fp32_refined"):
    # batches run the synchronous step (each step certified before the next), so
    # the solo runs they are compared with do too
    s = hc.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision=precision,
                  cg_rtol=w.cg_rtol, cg_maxit=2000, sync_cert=True)
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


def test_size_classes_of_the_sweep(hc):
    """The 48-instance sweep (16 each of 128^2, 256^2, 512^2, all refined)
    forms three size classes holding every instance; a double-float and an
    FP64 context stay on chains of their own."""
    ws = [W.sweep_instance(i) for i in range(48)]
    solvers = [solver_for(hc, w) for w in ws]
    extra = [solver_for(hc, W.sweep_instance(0), "fp64"),
             solver_for(hc, W.sweep_instance(1), "fp32_refined_df")]
    with hc.Batch(solvers + extra) as b:
        assert b.classes() == (3, 48)
        stats = b.step(1)
        assert all(x.status == 0 for x in stats)
    for s in solvers + extra:
        s.close()


def test_size_classes_match_solo_runs_bitwise(hc):
    """Members of batched size classes (two each of 128^2, 256^2 and 512^2,
    different c, D, gamma and m0) end bit-identical to their solo runs, as do
    an FP64 and a double-float context on chains of their own."""
    cases = [(0, "fp32_refined"), (3, "fp32_refined"), (1, "fp32_refined"), (4, "fp32_refined"),
             (2, "fp32_refined"), (47, "fp32_refined"), (13, "fp64"), (8, "fp32_refined_df")]
    ws = [W.sweep_instance(i) for i, _ in cases]
    solo = []
    for w, (i, prec) in zip(ws, cases):
        with solver_for(hc, w, prec) as s:
            st = s.step(3)
            solo.append((s.get_m(), s.get_p(), st.cg_iters, st.total_cg_iters))
    solvers = [solver_for(hc, w, prec) for w, (i, prec) in zip(ws, cases)]
    with hc.Batch(solvers) as b:
        assert b.classes() == (3, 6)
        stats = b.step(3)
    for s, st, (m, p, it, tot) in zip(solvers, stats, solo):
        assert st.status == 0
        assert np.array_equal(s.get_m(), m)
        assert np.array_equal(s.get_p(), p)
        assert st.cg_iters == it and st.total_cg_iters == tot
        s.close()


@pytest.mark.parametrize("n_idx", [0, 1, 2])
def test_size_class_members_follow_oracle(hc, n_idx):
    """One member of each size (128^2, 256^2, 512^2) in a class of three,
    four steps, against the FP64 oracle with the FP32-stored m and r: every
    step's certified residual recomputed with the oracle's operator (<= 1.2e-8,
    the refined bound with its rounding margin) and m within 1e-5.  A plain
    FP64 member of the same batch (a chain of its own) within 1e-9."""
    idx = [n_idx, n_idx + 3, n_idx + 6]
    ws = [W.sweep_instance(i) for i in idx]
    w = ws[0]
    g = O.Grid(w.n, w.L)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    prm = O.Params(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-12, cg_maxit=5000)
    w64 = W.sweep_instance(n_idx + 9)
    w64.cg_rtol = 1e-12  # both sides solve tightly: the FP64 bound is rounding, not the tolerance
    prm64 = O.Params(c=w64.c, D=w64.D, gamma=w64.gamma, dt=w64.dt, cg_rtol=w64.cg_rtol,
                     cg_maxit=2000)
    solvers = [solver_for(hc, x) for x in ws] + [solver_for(hc, w64, "fp64")]
    m, p = w.m0.copy(), np.zeros(g.shape)
    m64, p64 = w64.m0.copy(), np.zeros(g.shape)
    b_proj = O.project(g, w.S)
    with hc.Batch(solvers) as b:
        assert b.classes() == (1, 3)
        for k in range(4):
            # the GPU's state before the step, as the refined path holds it
            m_in = f32(solvers[0].get_m())
            stats = b.step(1)
            assert all(x.status == 0 for x in stats)
            p_gpu = solvers[0].get_p()
            res = np.linalg.norm(b_proj - O.apply_A(g, m_in, f32(w.r), p_gpu)) / np.linalg.norm(b_proj)
            assert stats[0].rel_residual <= w.cg_rtol and res <= 1.2e-8, (k, res)
            m, p, _ = O.step(g, prm, f32(w.r), w.S, f32(m), p)
            m64, p64, _ = O.step(g, prm64, w64.r, w64.S, m64, p64)
    assert rel_l2(solvers[0].get_m(), m) <= 1e-5
    assert rel_l2(solvers[3].get_m(), m64) <= 1e-9
    for s in solvers:
        s.close()
