"""Pins for the oracle's discrete adjoint: central finite differences of the
oracle's own forward map (Algorithm 1, several steps) in every input the
adjoint differentiates - c^2, D^2, r, S, m0 - on a ragged grid, for the three
relaxation branches (gamma < 1, gamma = 1, gamma > 1)."""
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
