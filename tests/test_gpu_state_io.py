"""hc_set_state / hc_get_state against the single-field calls, through the
C ABI: moving m and p in one call gives the same state, bit for bit, in every
precision mode and grid kind (2D powers of two, a mixed-radix 2D grid, 3D),
with numpy and page-locked torch buffers."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W
from gpu_common import hc  # noqa: F401

pytestmark = pytest.mark.gpu

# (64, 256) and (512, 512) refined: p crosses in four row pieces; the others in one
CASES = [((64, 256), "fp32_refined"), ((512, 512), "fp32_refined"),
         ((64, 32), "fp32_refined"), ((64, 32), "fp64"), ((64, 32), "fp32_refined_df"),
         ((2048, 16), "fp32_refined"), ((48, 40), "fp64"), ((16, 16, 16), "fp32_refined"),
         ((16, 8, 16), "fp64")]


def make(hc, n, precision):
    dim = len(n)
    L = (1.0,) * dim
    center = (0.3,) + (0.5,) * (dim - 1)
    center2 = (0.7,) + (0.5,) * (dim - 1)
    S = W.minus_mean(W.gaussian(n, center, 0.1, L) - W.gaussian(n, center2, 0.1, L))
    shape = tuple(reversed(n))
    s = hc.Solver(n, L, c=10.0, D=0.05, gamma=0.75, dt=1e-3, precision=precision,
                  cg_rtol=1e-9, cg_maxit=2000)
    s.set_r(W.smooth_r(n, 0, L))
    s.set_source(S)
    s.set_m(W.uniform_m(shape, dim, 0.0, 0.5, 0))
    return s


@pytest.mark.parametrize("n,precision", CASES)
def test_state_calls_match_single_field_calls(hc, n, precision):
    with make(hc, n, precision) as a, make(hc, n, precision) as b:
        a.step(2)
        b.step(2)
        # get: one call against get_m + get_p of the same state
        m1, p1 = a.get_state()
        assert np.array_equal(m1, a.get_m()) and np.array_equal(p1, a.get_p())
        # set: a perturbed state through set_state on one, set_m + set_p on the other
        rng = np.random.default_rng(1)
        m2 = m1 * (1.0 + 0.01 * rng.standard_normal(m1.shape))
        p2 = p1 + 0.01 * np.abs(p1).max() * rng.standard_normal(p1.shape)
        a.set_state(m2, p2)
        b.set_m(m2)
        b.set_p(p2)
        assert np.array_equal(a.get_m(), b.get_m()) and np.array_equal(a.get_p(), b.get_p())
        sa, sb = a.step(2), b.step(2)
        assert sa.total_cg_iters == sb.total_cg_iters
        ma, pa = a.get_state()
        assert np.array_equal(ma, b.get_m()) and np.array_equal(pa, b.get_p())


def test_state_calls_with_page_locked_buffers(hc):
    """The e2e pattern: page-locked torch buffers in and out every step, two
    steps in a row, against numpy buffers on a second context."""
    n = (256, 512)
    with make(hc, n, "fp32_refined") as a, make(hc, n, "fp32_refined") as b:
        a.step(1)
        b.step(1)
        npts = n[0] * n[1]
        hm = torch.empty(2 * npts, dtype=torch.float64, pin_memory=True)
        hp = torch.empty(npts, dtype=torch.float64, pin_memory=True)
        a.get_state(hm, hp)
        for _ in range(2):
            a.set_state(hm, hp)
            a.step(1)
            a.get_state(hm, hp)
            m, p = b.get_state()
            b.set_state(m, p)
            b.step(1)
        m, p = b.get_state()
        assert np.array_equal(hm.numpy().reshape(m.shape), m)
        assert np.array_equal(hp.numpy().reshape(p.shape), p)


def test_state_call_arguments(hc):
    """NULL buffers and wrong counts are rejected before any copy."""
    from paper_2606_06720_gb300 import _binding as B
    dp = C.POINTER(C.c_double)
    with make(hc, (32, 32), "fp32_refined") as s:
        m, p = s.get_state()
        pm, pp = m.ctypes.data_as(dp), p.ctypes.data_as(dp)
        assert B.hc_set_state(s.ctx, dp(), m.size, pp, p.size) == hc.HC_EINVAL
        assert B.hc_set_state(s.ctx, pm, m.size, pp, p.size + 1) == hc.HC_EINVAL
        assert B.hc_get_state(s.ctx, pm, m.size - 1, pp, p.size) == hc.HC_EINVAL
        assert B.hc_get_state(s.ctx, pm, m.size, dp(), p.size) == hc.HC_EINVAL
        m2, p2 = s.get_state()
        assert np.array_equal(m, m2) and np.array_equal(p, p2)
