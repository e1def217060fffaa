"""Repeatability at full size, as the stand-in for a race detector (the
memory checker's race tool may not run here).

Every kernel is deterministic by construction. Reductions go through per-CTA
partials summed in a fixed order by the last CTA, and the only atomics are
integer tickets. So two runs from identical inputs must agree bit for bit, and
a difference would point to a race. At full size the persistent column passes
hold several tiles per CTA and double-buffer them with asynchronous copies,
which is where a missing barrier would show.

Cases: the 2048² source/sink steps in each precision with the default launch
shapes; the FP32 refinement with the persistent column passes, the persistent
row pass, and both; and the 256³ refined steps."""
import numpy as np
import pytest

import workloads as W
from gpu_common import hc  # noqa: F401

pytestmark = pytest.mark.gpu


def run(hc, w, precision, nsteps, tuning=None):
    with hc.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision=precision,
                   cg_rtol=1e-8 if precision != "fp64" else 1e-10, cg_maxit=3000,
                   precond="kbar") as s:
        if tuning is not None:
            t = s.get_tuning()
            col = list(t["col_tile"])
            if tuning[0][0]:  # the persistent passes double-buffer tiles of at most 512 threads
                col[0] = min(col[0], 512 // (w.n[1] // 8))
            s.set_tuning(col, t["row_rows"], *tuning)
        s.set_r(w.r)
        s.set_source(w.S)
        s.set_m(w.m0)
        st = s.step(nsteps)
        return s.get_m(), s.get_p(), (st.total_cg_iters, st.total_sweeps, st.rel_residual)


# tuning = (col_pipe, row_pipe), [FP32 passes, FP64 passes]. At 2048² only the FP32 column
# passes may run persistent: the FP64 double buffer would not fit in shared memory.
@pytest.mark.parametrize("precision,tuning", [("fp32_refined", None), ("fp32_refined_df", None),
                                              ("fp64", None), ("fp32_refined", ([1, 0], [0, 0])),
                                              ("fp32_refined", ([0, 0], [1, 0])),
                                              ("fp32_refined", ([1, 0], [1, 0]))])
def test_2048_steps_repeat_bitwise(hc, precision, tuning):
    w = W.source_sink_2d(2048, steps=3)
    a = run(hc, w, precision, 3 if precision != "fp64" else 1, tuning)
    b = run(hc, w, precision, 3 if precision != "fp64" else 1, tuning)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2] == b[2]


def test_256_cubed_steps_repeat_bitwise(hc):
    w = W.source_sink_3d(256)
    a = run(hc, w, "fp32_refined", 2)
    b = run(hc, w, "fp32_refined", 2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2] == b[2]
