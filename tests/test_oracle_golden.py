"""Pins the oracle to closed-form values worked out by hand in
tests/golden/closed_forms.txt. That file gives each value with its arithmetic
and the equation it follows. The cases cover:

- the Fourier variables of Section 2.3.3, and the zeroed Nyquist derivative of reading R1;
- the spectral gradient inside eq. (p_discrete);
- activation in the projector form of eq. (m_activation_discrete);
- relaxation in every regime of eq. (m_relaxation_discrete);
- diffusion by eq. (diffusion_space_discrete), including the Nyquist wavenumber +pi N / L;
- the pressure operator and its solve, eq. (p_discrete), with constant, variable and cross
  coefficients, in 2D and 3D;
- the discrete energy E_h of Section 2.5;
- the preconditioner constants of reading R3: the scalar kappa and the matrix Kbar.

The expected numbers were computed by hand, not by a program, so they
are independent of the oracle's code. Trigonometric fields are evaluated on
the grid nodes x_i = i L / N."""
import math

import numpy as np
import pytest

import oracle as O
from golden_cases import CASES, field, num, of_kind, vec


def grid_of(d):
    n = tuple(int(x) for x in d["n"].split(","))
    L = tuple(num(x) for x in d["L"].split(","))
    return O.Grid(n, L), n, L


def test_every_kind_is_present():
    kinds = {c.values[0] for c in CASES}
    assert kinds == {"xi", "gradient", "activation", "relaxation", "diffusion", "pressure",
                     "energy", "kappa"}


@pytest.mark.parametrize("kind,d", of_kind("xi"))
def test_wavenumbers(kind, d):
    N, L = int(d["N"]), num(d["L"])
    for l, xi, xd in zip(d["l"].split(","), vec(d["xi"]), vec(d["xi_deriv"])):
        assert O.xi(int(l), N, L) == pytest.approx(xi, abs=1e-12)
        assert O.xi_deriv(int(l), N, L) == pytest.approx(xd, abs=1e-12)


@pytest.mark.parametrize("kind,d", of_kind("gradient"))
def test_gradient(kind, d):
    g, n, L = grid_of(d)
    out = O.gradient(g, field(d["f"], n, L))
    for a in range(len(n)):
        assert np.allclose(out[a], field(d[f"d{a}"], n, L), rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind,d", of_kind("activation"))
def test_activation(kind, d):
    m, gp, want = vec(d["m"]), vec(d["g"]), vec(d["expect"])
    out = O.activation(m.reshape(-1, 1), gp.reshape(-1, 1), num(d["c"]), num(d["dt"]))
    assert np.allclose(out[:, 0], want, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("kind,d", of_kind("relaxation"))
def test_relaxation(kind, d):
    m, want = vec(d["m"]), vec(d["expect"])
    out = O.relaxation(m.reshape(-1, 1), num(d["gamma"]), num(d["dt"]))
    assert np.allclose(out[:, 0], want, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("kind,d", of_kind("diffusion"))
def test_diffusion(kind, d):
    g, n, L = grid_of(d)
    m = np.stack([field(d[f"m{a}"], n, L) for a in range(len(n))])
    out = O.diffusion(g, m, num(d["D"]), num(d["dt"]))
    for a in range(len(n)):
        assert np.allclose(out[a], field(d[f"e{a}"], n, L), rtol=0, atol=1e-14)


@pytest.mark.parametrize("kind,d", of_kind("pressure"))
def test_pressure_operator_and_solve(kind, d):
    g, n, L = grid_of(d)
    m = np.stack([field(d[f"m{a}"], n, L) for a in range(len(n))])
    r = field(d["r"], n, L)
    S = field(d["S"], n, L)
    p = field(d["p"], n, L)
    # the operator itself maps the closed-form pressure onto the source
    assert np.allclose(O.apply_A(g, m, r, p), S, rtol=0, atol=1e-12)
    # and the solve recovers it, with either preconditioner
    for precond in (0, 1):
        x, st = O.pcg(g, m, r, S, rtol=1e-13, precond=precond)
        assert st.rc == 0
        assert np.allclose(x, p, rtol=0, atol=1e-11)


@pytest.mark.parametrize("kind,d", of_kind("kappa"))
def test_preconditioner_constants(kind, d):
    g, n, L = grid_of(d)
    m = np.stack([field(d[f"m{a}"], n, L) for a in range(len(n))])
    r = field(d["r"], n, L)
    assert O.kappa_default(g, m, r) == pytest.approx(num(d["kappa"]), rel=1e-13)
    assert np.allclose(O.kbar_default(g, m, r), vec(d["kbar"]), rtol=1e-13, atol=1e-15)
    # the solver reports the constant it used
    S = field("1:cos:1:" + ":".join(["1"] * (len(n) - 1)), n, L)
    for precond in (0, 1):
        _, st = O.pcg(g, m, r, S, rtol=1e-6, precond=precond)
        assert st.kappa == pytest.approx(num(d["kappa"]), rel=1e-13)


@pytest.mark.parametrize("kind,d", of_kind("energy"))
def test_energy(kind, d):
    g, n, L = grid_of(d)
    m = np.stack([field(d[f"m{a}"], n, L) for a in range(len(n))])
    prm = O.Params(c=num(d["c"]), D=num(d["D"]), gamma=num(d["gamma"]), dt=1e-3)
    r, p = field(d["r"], n, L), field(d["p"], n, L)
    E = O.energy(g, prm, r, m, p)
    assert E == pytest.approx(num(d["E"]), rel=1e-12)
    if "S" in d:  # the fixture's p is the pressure of its S
        assert np.allclose(O.apply_A(g, m, r, p), field(d["S"], n, L), rtol=0, atol=1e-12)


def test_number_and_field_grammar():
    """The fixture's own mini-grammar, on values with known results."""
    assert num("2*pi") == pytest.approx(2 * math.pi)
    assert num("-1*pi") == pytest.approx(-math.pi)
    assert num("4*ln(2)") == pytest.approx(4 * math.log(2))
    assert num("pi*pi/3") == pytest.approx(math.pi ** 2 / 3)
    assert num("2/3") == pytest.approx(2 / 3)
    assert num("sqrt(0.5)") == pytest.approx(math.sqrt(0.5))
    assert num("2*pi*pi+2*pi*pi*ln(2)") == pytest.approx(2 * math.pi ** 2 * (1 + math.log(2)))
    assert num("-inf") == -math.inf
    f = field("0.5,2:cos:1:0,1:sin:0:1", (4, 4), (2 * math.pi, 2 * math.pi))
    assert f.shape == (4, 4)
    # x runs along the last axis: f[j, i] = 0.5 + 2 cos(x_i) + sin(y_j)
    assert f[0, 1] == pytest.approx(0.5 + 2 * math.cos(math.pi / 2))
    assert f[1, 0] == pytest.approx(0.5 + 2 + math.sin(math.pi / 2))
