"""The CUDA path against the hand-worked closed forms of
tests/golden/closed_forms.txt, through the C ABI, with no oracle in between.

Each fixture kind reaches the GPU through the component that computes it:
- gradient: hc_set_p, then hc_gradient.
- pressure: hc_apply_operator maps the closed-form p onto S, and one hc_step from
  p = 0 solves for p, with either preconditioner.
- relaxation: hc_split_step with p = 0, so activation is the identity, and D = 0, so
  diffusion is too. Every node holds the fixture's vector.
- activation: hc_split_step with p = sum_a g_a sin(x_a) on [0, 2 pi]^d, so grad p =
  g at node 0. gamma = 1 makes relaxation the factor exp(-dt), and D = 0 leaves
  diffusion out.
- diffusion: hc_split_step with p = 0 and gamma = 1; relaxation contributes exp(-dt)
  again.
- kappa: the preconditioner constant the step reports.
- energy: the diagnostics energy E_h of a step's starting m, whose pressure the
  fixture's S gives.

The refined modes hold m and r in FP32 and compute the transforms in FP32, so
their bound is 1e-5 relative. FP64 keeps rounding-level bounds. The solves
run to a relative residual of 1e-12 (FP64) or 1e-10 (refined)."""
import math

import numpy as np
import pytest

from golden_cases import field, grid_dims, num, of_kind, vec, vector_field
from gpu_common import hc  # noqa: F401

pytestmark = pytest.mark.gpu

ALL = ["fp64", "fp32_refined", "fp32_refined_df"]
TWO = ["fp64", "fp32_refined"]       # the double-float mode shares the FP32 operator and split step
TOL = {"fp64": 1e-11, "fp32_refined": 1e-5, "fp32_refined_df": 1e-5}
SOLVE_TOL = {"fp64": 1e-9, "fp32_refined": 1e-5, "fp32_refined_df": 1e-5}
RTOL_CG = {"fp64": 1e-12, "fp32_refined": 1e-10, "fp32_refined_df": 1e-10}


def on_gpu_grid(d):
    """The library takes power-of-two axes of at least 8 nodes."""
    return all(v >= 8 for v in grid_dims(d)[0])


def close(got, want, tol):
    want = np.asarray(want, dtype=np.float64)
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(np.asarray(got) - want).max())
    assert err <= tol * scale, f"max error {err:.3e} > {tol:.1e} * {scale:.3g}"


def solver(hc, n, L, precision, **kw):
    args = dict(c=1.0, D=0.0, gamma=1.0, dt=1e-3)
    args.update(kw)
    return hc.Solver(n, L, precision=precision, **args)


@pytest.mark.parametrize("precision", ALL)
@pytest.mark.parametrize("kind,d", of_kind("gradient", on_gpu_grid))
def test_gradient(hc, precision, kind, d):
    n, L = grid_dims(d)
    with solver(hc, n, L, precision) as s:
        s.set_p(field(d["f"], n, L))
        got = s.gradient()
    close(got, vector_field(d, "d", n, L), TOL[precision])


@pytest.mark.parametrize("precision", TWO)
@pytest.mark.parametrize("kind,d", of_kind("pressure", on_gpu_grid))
def test_operator(hc, precision, kind, d):
    n, L = grid_dims(d)
    with solver(hc, n, L, precision) as s:
        s.set_r(field(d["r"], n, L))
        s.set_m(vector_field(d, "m", n, L))
        got = s.apply_operator(field(d["p"], n, L))
    close(got, field(d["S"], n, L), TOL[precision])


@pytest.mark.parametrize("precond", ["scalar", "kbar"])
@pytest.mark.parametrize("precision", ALL)
@pytest.mark.parametrize("kind,d", of_kind("pressure", on_gpu_grid))
def test_pressure_solve(hc, precision, precond, kind, d):
    n, L = grid_dims(d)
    with solver(hc, n, L, precision, cg_rtol=RTOL_CG[precision], precond=precond) as s:
        s.set_r(field(d["r"], n, L))
        s.set_m(vector_field(d, "m", n, L))
        s.set_source(field(d["S"], n, L))
        st = s.step(1)
        got = s.get_p()
    assert st.rc == 0
    close(got, field(d["p"], n, L), SOLVE_TOL[precision])


@pytest.mark.parametrize("precision", TWO)
@pytest.mark.parametrize("kind,d", of_kind("relaxation"))
def test_relaxation(hc, precision, kind, d):
    m, want = vec(d["m"]), vec(d["expect"])
    dim = len(m)
    n, L = (8,) * dim, (1.0,) * dim
    shape = (8,) * dim
    with solver(hc, n, L, precision, gamma=num(d["gamma"]), dt=num(d["dt"])) as s:
        s.set_p(np.zeros(shape))
        s.set_m(np.broadcast_to(m.reshape((dim,) + (1,) * dim), (dim,) + shape))
        s.split_step()
        got = s.get_m()
    close(got, np.broadcast_to(want.reshape((dim,) + (1,) * dim), (dim,) + shape), TOL[precision])


@pytest.mark.parametrize("precision", TWO)
@pytest.mark.parametrize("kind,d", of_kind("activation"))
def test_activation(hc, precision, kind, d):
    m, g, want = vec(d["m"]), vec(d["g"]), vec(d["expect"])
    dim = len(m)
    n, L = (8,) * dim, (2 * math.pi,) * dim
    shape = (8,) * dim
    # p = sum_a g_a sin(x_a): grad p = (g_a cos x_a), equal to g at node 0
    p = sum(float(g[a]) * field(f"1:sin:{':'.join('1' if b == a else '0' for b in range(dim))}", n, L)
            for a in range(dim))
    dt = num(d["dt"])
    with solver(hc, n, L, precision, c=num(d["c"]), gamma=1.0, dt=dt) as s:
        s.set_p(p)
        s.set_m(np.broadcast_to(m.reshape((dim,) + (1,) * dim), (dim,) + shape))
        s.split_step()
        got = s.get_m()
    node0 = got[(slice(None),) + (0,) * dim]
    close(node0, want * math.exp(-dt), TOL[precision])


@pytest.mark.parametrize("precision", TWO)
@pytest.mark.parametrize("kind,d", of_kind("diffusion", on_gpu_grid))
def test_diffusion(hc, precision, kind, d):
    n, L = grid_dims(d)
    dt = num(d["dt"])
    with solver(hc, n, L, precision, D=num(d["D"]), gamma=1.0, dt=dt) as s:
        s.set_p(np.zeros(tuple(reversed(n))))
        s.set_m(vector_field(d, "m", n, L))
        s.split_step()
        got = s.get_m()
    close(got, vector_field(d, "e", n, L) * math.exp(-dt), TOL[precision])


@pytest.mark.parametrize("precond", ["scalar", "kbar"])
@pytest.mark.parametrize("precision", ALL)
@pytest.mark.parametrize("kind,d", of_kind("kappa", on_gpu_grid))
def test_preconditioner_constant(hc, precision, precond, kind, d):
    n, L = grid_dims(d)
    S = field("1:cos:" + ":".join(["1"] * len(n)), n, L)
    with solver(hc, n, L, precision, cg_rtol=1e-6, precond=precond) as s:
        s.set_r(field(d["r"], n, L))
        s.set_m(vector_field(d, "m", n, L))
        s.set_source(S)
        st = s.step(1)
    assert st.kappa == pytest.approx(num(d["kappa"]), rel=TOL[precision])


@pytest.mark.parametrize("precision", ALL)
@pytest.mark.parametrize("kind,d", of_kind("energy", lambda d: "S" in d and on_gpu_grid(d)))
def test_energy(hc, precision, kind, d):
    n, L = grid_dims(d)
    with solver(hc, n, L, precision, c=num(d["c"]), D=num(d["D"]), gamma=num(d["gamma"]),
                cg_rtol=RTOL_CG[precision], diagnostics=True) as s:
        s.set_r(field(d["r"], n, L))
        s.set_m(vector_field(d, "m", n, L))
        s.set_source(field(d["S"], n, L))
        st = s.step(1)
    assert st.energy_valid == 1
    assert st.energy == pytest.approx(num(d["E"]), rel=SOLVE_TOL[precision])
