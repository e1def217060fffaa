"""Reader of tests/golden/closed_forms.txt, the hand-worked closed-form values
that pin both the oracle and the GPU path (pure parsing; none of the scheme's
arithmetic). The file's header describes its format."""
import math
import os
import re

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "closed_forms.txt")


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


def _product(tok: str) -> float:
    parts = re.split(r"([*/])", tok.strip())
    v = _factor(parts[0])
    for op, f in zip(parts[1::2], parts[2::2]):
        v = v * _factor(f) if op == "*" else v / _factor(f)
    return v


def num(tok: str) -> float:
    """A sum of products or quotients of factors: decimals, pi, ln(k),
    sqrt(k), inf."""
    return sum(_product(t) for t in tok.strip().split("+"))


def vec(tok: str) -> np.ndarray:
    return np.array([num(t) for t in tok.split(",")])


def coords(n, L):
    """Node coordinates x_i = i L / N, one array per axis, in the (.., y, x) layout."""
    axes = [np.arange(N) * (Lx / N) for N, Lx in zip(n, L)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return grids[::-1]


def field(spec: str, n, L) -> np.ndarray:
    """Sum of constants and terms amp:trig:k1:k2[:k3] on the grid."""
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


def vector_field(d: dict, prefix: str, n, L) -> np.ndarray:
    return np.stack([field(d[f"{prefix}{a}"], n, L) for a in range(len(n))])


def grid_dims(d: dict):
    n = tuple(int(x) for x in d["n"].split(","))
    L = tuple(num(x) for x in d["L"].split(","))
    return n, L


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


def of_kind(kind, keep=None):
    """The cases of one kind, optionally filtered by keep(d)."""
    return [c for c in CASES if c.values[0] == kind and (keep is None or keep(c.values[1]))]
