"""Seeded synthetic inputs for the Hu-Cai step: conductivity fields m0,
permeability fields r and source/sink fields S, on uniform periodic grids.

This module is the one piece shared by the oracle side (tests) and the GPU
side (tests, bench).  It generates inputs only and holds none of the scheme's
arithmetic: no transforms, no operator, no solver, no substep.

Field conventions: 2D scalar fields have numpy shape ``(ny, nx)``, 3D
``(nz, ny, nx)``, x fastest; vector fields carry a leading component axis.
Nodes sit at x_i = i L / N, the periodic end point excluded.

Recipes (all inputs of the paper's experiments are analytic, Section 3.1):
  * ``uniform_m``: iid uniform components from ``numpy.random.default_rng(seed)``.
  * ``gaussian``: exp(-|x - x0|^2 / (2 sigma^2)) with the minimum-image
    periodic distance.
  * ``smooth_field``: real trigonometric polynomial over integer wavevectors
    0 < |k| <= kmax (half-space representatives, lexicographic order), with
    coefficients a_k, b_k ~ N(0,1) from the seed, scaled so that its maximum
    modulus on a fixed 256^d sampling lattice is 1.  It is evaluated exactly at
    the nodes, so the same seed gives the same continuous field at every
    resolution.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


def node_coords(n: int, L: float = 1.0) -> np.ndarray:
    return np.arange(n, dtype=np.float64) * (L / n)


def uniform_m(shape: tuple, dim: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(dim,) + tuple(shape))


def gaussian(n: tuple, center: tuple, sigma: float, L: tuple | None = None) -> np.ndarray:
    """exp(-d^2/(2 sigma^2)), d the periodic minimum-image distance to ``center``.
    ``n = (nx, ny[, nz])``; returns shape reversed(n)."""
    L = L or tuple(1.0 for _ in n)
    d2 = 0.0
    axes = []
    for a, (na, La, ca) in enumerate(zip(n, L, center)):
        x = node_coords(na, La) - ca
        x = x - La * np.round(x / La)
        axes.append(x * x)
    # broadcast: axis a of n is numpy axis (dim-1-a)
    dim = len(n)
    for a in range(dim):
        shp = [1] * dim
        shp[dim - 1 - a] = n[a]
        d2 = d2 + axes[a].reshape(shp)
    return np.exp(-d2 / (2.0 * sigma * sigma))


def _wavevectors(dim: int, kmax: int):
    """Half-space representatives k != 0, |k| <= kmax, lexicographic in (kx, ky[, kz])."""
    out = []
    rng = range(-kmax, kmax + 1)
    for k in itertools.product(rng, repeat=dim):
        if sum(c * c for c in k) == 0 or sum(c * c for c in k) > kmax * kmax:
            continue
        # first nonzero component positive
        first = next(c for c in k if c != 0)
        if first > 0:
            out.append(k)
    return out


def _trig_poly(n: tuple, L: tuple, ks, coef) -> np.ndarray:
    """Re sum_k coef_k exp(2 pi i k . x / L) at the nodes, by separable sums."""
    dim = len(n)
    kmax = max(max(abs(c) for c in k) for k in ks)
    span = 2 * kmax + 1
    E = [np.exp(2j * np.pi * np.outer(node_coords(n[a], L[a]) / L[a], np.arange(-kmax, kmax + 1)))
         for a in range(dim)]  # E[a][i, k + kmax]
    C = np.zeros((span,) * dim, dtype=np.complex128)  # indexed [kx, ky(, kz)]
    for k, c in zip(ks, coef):
        C[tuple(kk + kmax for kk in k)] += c
    if dim == 2:
        # f[j, i] = sum_{kx,ky} C[kx,ky] Ex[i,kx] Ey[j,ky]
        f = E[1] @ (E[0] @ C).T
    else:
        f = np.einsum("ia,jb,kc,abc->kji", E[0], E[1], E[2], C, optimize=True)
    return f.real


def smooth_field(n: tuple, seed: int, kmax: int = 8, L: tuple | None = None) -> np.ndarray:
    L = L or tuple(1.0 for _ in n)
    dim = len(n)
    ks = _wavevectors(dim, kmax)
    rng = np.random.default_rng(seed)
    ab = rng.standard_normal((len(ks), 2))
    coef = ab[:, 0] - 1j * ab[:, 1]  # a cos + b sin = Re((a - i b) e^{i theta})
    ref = _trig_poly(tuple(256 for _ in n) if dim == 2 else tuple(64 for _ in n), L, ks, coef)
    scale = 1.0 / np.abs(ref).max()
    return _trig_poly(n, L, ks, coef) * scale


def smooth_r(n: tuple, seed: int = 0, L: tuple | None = None) -> np.ndarray:
    """r = max(0.1 + 0.05 f, 0.05), f the seeded smooth field, so r in [0.05, 0.15]."""
    return np.maximum(0.1 + 0.05 * smooth_field(n, seed, 8, L), 0.05)


def minus_mean(f: np.ndarray) -> np.ndarray:
    return f - f.mean()


@dataclass
class Workload:
    """A named synthetic problem: grid, model parameters and initial fields."""
    name: str
    n: tuple
    L: tuple
    c: float
    D: float
    gamma: float
    dt: float
    steps: int
    cg_rtol: float
    r: np.ndarray = field(repr=False)
    S: np.ndarray = field(repr=False)
    m0: np.ndarray = field(repr=False)

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def shape(self) -> tuple:
        return tuple(reversed(self.n))

    @property
    def npts(self) -> int:
        return int(np.prod(self.n))


def centered_gaussian_2d(n: int) -> Workload:
    """64^2-style problem: r = 0.1, S = centred Gaussian (sigma 0.05) minus its
    mean, m0 ~ U[0,1] (seed 0), c=10, D=0.05, gamma=0.75, dt=1e-3, rtol 1e-10."""
    nn = (n, n)
    S = minus_mean(gaussian(nn, (0.5, 0.5), 0.05))
    return Workload("gauss_center_%d" % n, nn, (1.0, 1.0), 10.0, 0.05, 0.75, 1e-3, 100, 1e-10,
                    np.full((n, n), 0.1), S, uniform_m((n, n), 2, 0.0, 1.0, 0))


def source_sink_2d(n: int, steps: int = 2000, gamma: float = 0.5, seed: int = 0) -> Workload:
    """512^2 / 2048^2 problem: smooth random r (seed 0) in [0.05, 0.15], S =
    +G(0.3,0.5) - G(0.7,0.5) (sigma 0.05) minus mean, m0 ~ U[0,0.5] (seed),
    c=25, D=0.02, gamma=0.5, dt=5e-4."""
    nn = (n, n)
    S = minus_mean(gaussian(nn, (0.3, 0.5), 0.05) - gaussian(nn, (0.7, 0.5), 0.05))
    return Workload("source_sink_%d" % n, nn, (1.0, 1.0), 25.0, 0.02, gamma, 5e-4, steps, 1e-8,
                    smooth_r(nn, 0), S, uniform_m((n, n), 2, 0.0, 0.5, seed))


SWEEP_C = (5.0, 10.0, 25.0, 50.0)
SWEEP_D = (0.01, 0.02, 0.05, 0.1)
SWEEP_GAMMA = (0.5, 0.75, 1.0)
SWEEP_SIZES = (128, 256, 512)


def sweep_instance(i: int) -> Workload:
    """Instance i (0..47) of the batched parameter sweep: the i-th (c, D, gamma)
    triple in lexicographic order, grid size SWEEP_SIZES[i % 3], r = 0.1,
    centred Gaussian S (sigma 0.05) minus mean, m0 ~ U[0,1] with seed i, dt=1e-3."""
    c, D, gamma = list(itertools.product(SWEEP_C, SWEEP_D, SWEEP_GAMMA))[i]
    n = SWEEP_SIZES[i % 3]
    nn = (n, n)
    S = minus_mean(gaussian(nn, (0.5, 0.5), 0.05))
    return Workload("sweep_%02d_%d" % (i, n), nn, (1.0, 1.0), c, D, gamma, 1e-3, 1000, 1e-8,
                    np.full((n, n), 0.1), S, uniform_m((n, n), 2, 0.0, 1.0, i))


def source_sink_3d(n: int, steps: int = 500) -> Workload:
    """3D problem: r = 0.1, S = +G(0.3,0.5,0.5) - G(0.7,0.5,0.5) (sigma 0.05)
    minus mean, m0 ~ U[0,0.5] per component (seed 0), c=25, D=0.03,
    gamma=0.75, dt=5e-4."""
    nn = (n, n, n)
    S = minus_mean(gaussian(nn, (0.3, 0.5, 0.5), 0.05) - gaussian(nn, (0.7, 0.5, 0.5), 0.05))
    return Workload("source_sink_3d_%d" % n, nn, (1.0, 1.0, 1.0), 25.0, 0.03, 0.75, 5e-4, steps,
                    1e-8, np.full((n, n, n), 0.1), S, uniform_m((n, n, n), 3, 0.0, 0.5, 0))


# ---------------------------------------------------------------- the paper's analytic inputs
# Section 3.1 (initial conductivities m^A, m^B, m^const), Section 3.2 (one
# source and four sinks, S_4) and Section 3.3 (internal sink, S_int), on the
# unit square, evaluated as printed at the nodes x_i = i / N (no periodic
# image: the Gaussians of S are below 1e-100 at the boundary; m^A is 3.7e-6
# there, which the paper treats as periodic).

def _xy(n: int):
    x = node_coords(n)
    return np.meshgrid(x, x)  # X[j, i] = x_i, Y[j, i] = y_j


def paper_m_ini(n: int, kind: str) -> np.ndarray:
    """m^A = (exp(-1e4 (y-0.5)^2 - 50 (x-0.5)^2), 0), m^B = (exp(-50 (y-0.5)^2
    - 50 (x-0.5)^2), 0), m^const = (1, 1); shape (2, n, n)."""
    X, Y = _xy(n)
    if kind == "A":
        m1 = np.exp(-1e4 * (Y - 0.5) ** 2 - 50.0 * (X - 0.5) ** 2)
    elif kind == "B":
        m1 = np.exp(-50.0 * (Y - 0.5) ** 2 - 50.0 * (X - 0.5) ** 2)
    elif kind == "const":
        return np.ones((2, n, n))
    else:
        raise ValueError(kind)
    return np.stack([m1, np.zeros_like(m1)])


def paper_S4(n: int) -> np.ndarray:
    """S_4 = exp(-1000 |x - (0.5,0.5)|^2) - sum_i exp(-1000 |x - x_i|^2) / 4,
    sinks at (0.2,0.2), (0.2,0.8), (0.8,0.2), (0.8,0.8)."""
    X, Y = _xy(n)
    S = np.exp(-1000.0 * ((Y - 0.5) ** 2 + (X - 0.5) ** 2))
    for xi, yi in ((0.2, 0.2), (0.2, 0.8), (0.8, 0.2), (0.8, 0.8)):
        S = S - 0.25 * np.exp(-1000.0 * ((Y - yi) ** 2 + (X - xi) ** 2))
    return S


def paper_Sint(n: int) -> np.ndarray:
    """S_int = exp(-1000 |x - (0.5,0.5)|^2) - pi / 1000."""
    X, Y = _xy(n)
    return np.exp(-1000.0 * ((Y - 0.5) ** 2 + (X - 0.5) ** 2)) - math.pi / 1000.0


def paper_four_sinks(n: int, gamma: float = 1.0, steps: int = 30000) -> Workload:
    """Section 3.2: r = 0.1, c = 200, D = 0.0025, dt = 0.005, S_4, m^A
    (t_end = 150); CG threshold 1e-7 and Delta m <= 1e-4 (Section 3.1)."""
    return Workload("paper_four_sinks_%d_g%g" % (n, gamma), (n, n), (1.0, 1.0), 200.0, 0.0025,
                    gamma, 0.005, steps, 1e-7, np.full((n, n), 0.1), paper_S4(n),
                    paper_m_ini(n, "A"))


def paper_internal_sink(n: int, gamma: float = 0.75, kind: str = "const",
                        steps: int = 40000) -> Workload:
    """Section 3.3: r = 0.1, c = 200, D = 0.0025, dt = 0.005, S_int, m^const
    (or m^A / m^B, Section 3.3's comparison at t = 200)."""
    return Workload("paper_internal_sink_%d_%s" % (n, kind), (n, n), (1.0, 1.0), 200.0, 0.0025,
                    gamma, 0.005, steps, 1e-7, np.full((n, n), 0.1), paper_Sint(n),
                    paper_m_ini(n, kind))


def paper_convergence(n: int, steps: int = 100) -> Workload:
    """Section 4's grid-convergence setup of its first table: Omega = [0,1]^2,
    N x N with N in {50, 100, 200, 400}, r = 0.1, S_int, m^A, c = 100,
    gamma = 0.75, D = 0.01, dt = 0.05 (steps = 100 reaches t = 5), CG threshold
    1e-7 (the paper's default, Section 3.1)."""
    return Workload("paper_convergence_%d" % n, (n, n), (1.0, 1.0), 100.0, 0.01, 0.75, 0.05, steps,
                    1e-7, np.full((n, n), 0.1), paper_Sint(n), paper_m_ini(n, "A"))
