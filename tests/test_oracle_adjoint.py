"""Pins for the oracle's discrete adjoint: finite differences of the oracle's
own forward map (Algorithm 1, several steps) in every input the adjoint
differentiates: c^2, D^2, r, S, m0. The cases cover:
- a ragged 2D grid and a 3D grid;
- the three relaxation branches (gamma < 1, gamma = 1, gamma > 1);
- the relaxation Jacobian's special points (m = 0, extinction);
- activation exponents on both sides of the switch between the series and
  the closed form of phi_1';
- c = 0, with a one-sided difference in c^2."""
import numpy as np
import pytest

import oracle as O
import workloads as W

RNG = np.random.default_rng(17)


def problem(gamma):
    n, L = (16, 8), (1.0, 0.5)
    g = O.Grid(n, L)
    X, Y = np.meshgrid(np.arange(16) / 16, np.arange(8) * 0.5 / 8)
    m0 = np.stack([0.5 + 0.2 * np.cos(2 * np.pi * X) + 0.05 * RNG.standard_normal(g.shape),
                   0.4 + 0.1 * np.sin(4 * np.pi * Y) + 0.05 * RNG.standard_normal(g.shape)])
    r = W.smooth_r(n, 2, L)
    S = W.minus_mean(W.gaussian(n, (0.3, 0.25), 0.08, L) - W.gaussian(n, (0.7, 0.25), 0.08, L))
    prm = O.Params(c=3.0, D=0.08, gamma=gamma, dt=2e-3, cg_rtol=1e-14, cg_maxit=3000)
    return g, prm, r, S, m0


def loss(g, prm, r, S, m0, w, nsteps):
    m, p = m0.copy(), np.zeros(g.shape)
    for _ in range(nsteps):
        m, p, st = O.step(g, prm, r, S, m, p)
    return float((w * m).sum())


@pytest.mark.parametrize("gamma", [0.75, 1.0, 1.5])
def test_adjoint_matches_central_differences(gamma):
    g, prm, r, S, m0 = problem(gamma)
    nsteps = 3
    w = RNG.standard_normal(m0.shape)
    adj = O.adjoint(g, prm, r, S, m0, np.zeros(g.shape), nsteps, w)

    def fd(f, h):
        return (f(h) - f(-h)) / (2 * h)

    def with_params(**kw):
        q = O.Params(**{**prm.__dict__, **kw})
        return q

    c2 = prm.c ** 2
    d_c2 = fd(lambda h: loss(g, with_params(c=np.sqrt(c2 + h)), r, S, m0, w, nsteps), 1e-4 * c2)
    assert np.isclose(adj["dc2"], d_c2, rtol=2e-6), (adj["dc2"], d_c2)
    D2 = prm.D ** 2
    d_D2 = fd(lambda h: loss(g, with_params(D=np.sqrt(D2 + h)), r, S, m0, w, nsteps), 1e-3 * D2)
    assert np.isclose(adj["dD2"], d_D2, rtol=2e-6), (adj["dD2"], d_D2)
    for (j, i) in [(1, 3), (5, 12), (6, 0)]:
        def pr(h, j=j, i=i):
            rr = r.copy(); rr[j, i] += h
            return loss(g, prm, rr, S, m0, w, nsteps)

        def ps(h, j=j, i=i):
            ss = S.copy(); ss[j, i] += h
            return loss(g, prm, r, ss, m0, w, nsteps)

        def pm(h, j=j, i=i, c=(i + j) % 2):
            mm = m0.copy(); mm[c, j, i] += h
            return loss(g, prm, r, S, mm, w, nsteps)

        scale = max(abs(adj["dr"]).max(), 1e-300)
        assert abs(adj["dr"][j, i] - fd(pr, 1e-5)) <= 1e-6 * scale
        scale = max(abs(adj["dS"]).max(), 1e-300)
        assert abs(adj["dS"][j, i] - fd(ps, 1e-5)) <= 1e-6 * scale
        c = (i + j) % 2
        scale = max(abs(adj["dm0"]).max(), 1e-300)
        assert abs(adj["dm0"][c, j, i] - fd(pm, 1e-6)) <= 1e-6 * scale


def test_adjoint_of_zero_steps_is_identity():
    g, prm, r, S, m0 = problem(0.75)
    w = RNG.standard_normal(m0.shape)
    adj = O.adjoint(g, prm, r, S, m0, np.zeros(g.shape), 0, w)
    assert np.array_equal(adj["dm0"], w)
    assert adj["dc2"] == 0 and adj["dD2"] == 0
    assert not adj["dr"].any() and not adj["dS"].any()


def test_adjoint_source_gradient_is_projected():
    """S enters only through its null-space projection (R2), so dL/dS has no
    corner-mode content: shifting S by a constant changes nothing."""
    g, prm, r, S, m0 = problem(0.75)
    w = RNG.standard_normal(m0.shape)
    adj = O.adjoint(g, prm, r, S, m0, np.zeros(g.shape), 2, w)
    assert abs(adj["dS"].sum()) < 1e-12 * abs(adj["dS"]).sum()
    assert np.allclose(O.project(g, adj["dS"]), adj["dS"], atol=1e-15)


def fd_central(f, h):
    return (f(h) - f(-h)) / (2 * h)


def check_fields(g, prm, r, S, m0, w, nsteps, adj, points, comps=None):
    """Central differences of the loss in r, S and m0 at the given points."""
    dim = m0.shape[0]
    for k, idx in enumerate(points):
        def pr(h, idx=idx):
            rr = r.copy(); rr[idx] += h
            return loss(g, prm, rr, S, m0, w, nsteps)

        def ps(h, idx=idx):
            ss = S.copy(); ss[idx] += h
            return loss(g, prm, r, ss, m0, w, nsteps)

        c = comps[k] if comps is not None else k % dim

        def pm(h, idx=idx, c=c):
            mm = m0.copy(); mm[(c,) + idx] += h
            return loss(g, prm, r, S, mm, w, nsteps)

        for key, f, h, at in (("dr", pr, 1e-5, idx), ("dS", ps, 1e-5, idx),
                              ("dm0", pm, 1e-6, (c,) + idx)):
            scale = max(abs(adj[key]).max(), 1e-300)
            assert abs(adj[key][at] - fd_central(f, h)) <= 1e-6 * scale, (key, at)


@pytest.mark.parametrize("gamma", [0.5, 1.5])
def test_adjoint_at_extinct_and_zero_conductivity(gamma):
    """The relaxation Jacobian's special points: m = 0 exactly (the map is
    the identity to first order for gamma > 1 and locally zero for gamma < 1),
    and for gamma < 1 points that die out in one step (|m| < dt: b < 0, the
    map is locally zero). The perturbations stay well inside each regime."""
    g, prm, r, S, m0 = problem(gamma)
    zero, extinct = [(2, 5), (6, 9)], [(4, 1), (1, 14)]
    for j, i in zero:
        m0[:, j, i] = 0.0
    for j, i in extinct:
        m0[:, j, i] = (0.3 * prm.dt, -0.2 * prm.dt)
    nsteps = 3
    w = RNG.standard_normal(m0.shape)
    adj = O.adjoint(g, prm, r, S, m0, np.zeros(g.shape), nsteps, w)
    if gamma < 1:
        # the local path is zero there; at m = 0 the pressure path (through
        # K = m m^T + r I) is zero too, at the extinct points it scales with |m| ~ dt
        for j, i in zero:
            assert not adj["dm0"][:, j, i].any()
        for j, i in extinct:
            assert np.abs(adj["dm0"][:, j, i]).max() < 1e-5 * np.abs(adj["dm0"]).max()
    check_fields(g, prm, r, S, m0, w, nsteps, adj, zero + extinct, comps=[0, 1, 0, 1])


def test_adjoint_with_large_activation_exponents():
    """c large enough that c^2 dt |grad p|^2 passes 0.5 at some points, where
    the derivative of phi_1 takes its closed form instead of its series."""
    g, prm, r, S, m0 = problem(0.75)
    _, p1, _ = O.step(g, prm, r, S, m0.copy(), np.zeros(g.shape))
    g2 = (O.gradient(g, p1) ** 2).sum(0)
    c = float(np.sqrt(2.0 / (prm.dt * g2.max())))   # largest exponent about 2
    prm = O.Params(**{**prm.__dict__, "c": c})
    z = c * c * prm.dt * g2
    assert (z > 0.5).any() and (z < 0.5).any()
    nsteps = 2
    w = RNG.standard_normal(m0.shape)
    adj = O.adjoint(g, prm, r, S, m0, np.zeros(g.shape), nsteps, w)
    c2 = c * c
    d_c2 = fd_central(lambda h: loss(g, O.Params(**{**prm.__dict__, "c": np.sqrt(c2 + h)}),
                                     r, S, m0, w, nsteps), 1e-5 * c2)
    assert np.isclose(adj["dc2"], d_c2, rtol=1e-5), (adj["dc2"], d_c2)
    j, i = np.unravel_index(np.argmax(z), z.shape)
    check_fields(g, prm, r, S, m0, w, nsteps, adj, [(int(j), int(i)), (3, 3)])


def test_adjoint_in_c2_at_zero_activation():
    """At c = 0 the activation is off, and dL/dc^2 is the first-order effect of
    switching it on: phi_1(0) = 1. c^2 cannot go below 0, so the derivative is
    taken one-sided, to second order: (-3 L(0) + 4 L(h) - L(2h)) / (2h)."""
    g, prm, r, S, m0 = problem(0.75)
    prm = O.Params(**{**prm.__dict__, "c": 0.0})
    nsteps = 2
    w = RNG.standard_normal(m0.shape)
    adj = O.adjoint(g, prm, r, S, m0, np.zeros(g.shape), nsteps, w)

    def L(c2):
        return loss(g, O.Params(**{**prm.__dict__, "c": np.sqrt(c2)}), r, S, m0, w, nsteps)

    h = 1e-3
    d_c2 = (-3 * L(0.0) + 4 * L(h) - L(2 * h)) / (2 * h)
    assert abs(adj["dc2"]) > 0
    assert np.isclose(adj["dc2"], d_c2, rtol=1e-5), (adj["dc2"], d_c2)


def test_adjoint_3d_matches_central_differences():
    """The oracle's adjoint on a 3D grid (x, y, z components of m and grad p)."""
    n, L = (8, 8, 8), (1.0, 1.0, 0.5)
    g = O.Grid(n, L)
    r = 0.1 + 0.02 * RNG.uniform(0, 1, g.shape)
    S = W.minus_mean(RNG.standard_normal(g.shape))
    m0 = 0.4 + 0.1 * RNG.standard_normal((3,) + g.shape)
    prm = O.Params(c=2.0, D=0.08, gamma=0.75, dt=2e-3, cg_rtol=1e-14, cg_maxit=3000)
    nsteps = 2
    w = RNG.standard_normal(m0.shape)
    adj = O.adjoint(g, prm, r, S, m0, np.zeros(g.shape), nsteps, w)
    c2 = prm.c ** 2
    d_c2 = fd_central(lambda h: loss(g, O.Params(**{**prm.__dict__, "c": np.sqrt(c2 + h)}),
                                     r, S, m0, w, nsteps), 1e-4 * c2)
    assert np.isclose(adj["dc2"], d_c2, rtol=2e-6), (adj["dc2"], d_c2)
    D2 = prm.D ** 2
    d_D2 = fd_central(lambda h: loss(g, O.Params(**{**prm.__dict__, "D": np.sqrt(D2 + h)}),
                                     r, S, m0, w, nsteps), 1e-3 * D2)
    assert np.isclose(adj["dD2"], d_D2, rtol=2e-6), (adj["dD2"], d_D2)
    check_fields(g, prm, r, S, m0, w, nsteps, adj, [(1, 2, 3), (5, 0, 7), (7, 6, 1)],
                 comps=[0, 1, 2])
