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
import os
import re

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")


def _factor(tok: str) -> float:
    neg = tok.startswith("-")
    t = tok[1:] if neg else tok
    if t == "pi":
        v = math.pi
    elif (mt := re.fullmatch(r"ln\(([0-9.]+)\)", t)):
        v = math.log(float(mt.group(1)))
    elif (mt := re.fullmatch(r"sqrt\(([0-9.]+)\)", t)):
        v = math.sqrt(float(mt.group(1)))
    else:
        v = float(t)
    return -v if neg else v


def num(tok: str) -> float:
    parts = re.split(r"([*/])", tok.strip())
    v = _factor(parts[0])
    for op, f in zip(parts[1::2], parts[2::2]):
        v = v * _factor(f) if op == "*" else v / _factor(f)
    return v


def vec(tok: str) -> np.ndarray:
    return np.array([num(t) for t in tok.split(",")])


def coords(n, L):
    """Node coordinates, one array per axis, in the oracle's (.., y, x) layout."""
    axes = [np.arange(N) * (Lx / N) for N, Lx in zip(n, L)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return grids[::-1]


def field(spec: str, n, L) -> np.ndarray:
    X = coords(n, L)
    out = np.zeros(X[0].shape)
    for term in spec.split(","):
        if ":" not in term:
            out += num(term)
            continue
        amp, trig, *k = term.split(":")
        assert trig in ("cos", "sin") and len(k) == len(n)
        arg = sum(2 * math.pi * int(ka) * Xa / La for ka, Xa, La in zip(k, X, L))
        out += num(amp) * (np.cos(arg) if trig == "cos" else np.sin(arg))
    return out


def load_cases():
    cases = []
    with open(GOLDEN) as f:
        for lineno, line in enumerate(f, 1):
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, *kv = [s.strip() for s in line.split(";")]
            d = dict(s.split("=", 1) for s in kv)
            assert "cite" in d, f"line {lineno} cites no passage"
            cases.append(pytest.param(kind, d, id=f"{kind}-line{lineno}"))
    return cases


CASES = load_cases()


def of_kind(kind):
    return [c for c in CASES if c.values[0] == kind]


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
    E = O.energy(g, prm, field(d["r"], n, L), m, field(d["p"], n, L))
    assert E == pytest.approx(num(d["E"]), rel=1e-12)


def test_number_and_field_grammar():
    """The fixture's own mini-grammar, on values with known results."""
    assert num("2*pi") == pytest.approx(2 * math.pi)
    assert num("-1*pi") == pytest.approx(-math.pi)
    assert num("4*ln(2)") == pytest.approx(4 * math.log(2))
    assert num("pi*pi/3") == pytest.approx(math.pi ** 2 / 3)
    assert num("2/3") == pytest.approx(2 / 3)
    assert num("sqrt(0.5)") == pytest.approx(math.sqrt(0.5))
    f = field("0.5,2:cos:1:0,1:sin:0:1", (4, 4), (2 * math.pi, 2 * math.pi))
    assert f.shape == (4, 4)
    # x runs along the last axis: f[j, i] = 0.5 + 2 cos(x_i) + sin(y_j)
    assert f[0, 1] == pytest.approx(0.5 + 2 * math.cos(math.pi / 2))
    assert f[1, 0] == pytest.approx(0.5 + 2 + math.sin(math.pi / 2))
