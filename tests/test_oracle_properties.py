"""Properties that the mathematics fixes for any grid and any fields, checked
on the oracle with randomly drawn sizes (odd and even, 2D and 3D) and values:

- Transforms: the inverse transform undoes the forward one, and Parseval's
  identity holds.
- Operator of eq. (p_discrete): symmetric, positive semi-definite, and blind to
  the null space (A P = A, with P the projection of reading R2).
- Projection: idempotent, and orthogonal.
- Relaxation, eq. (m_relaxation_discrete): keeps the direction of m and never
  grows |m| (gamma > 0).
- Activation, eq. (m_activation_discrete): leaves the part of m across grad p
  unchanged and never shrinks the part along it.
- Diffusion, eq. (diffusion_space_discrete): keeps the mean of each component
  and never grows its L2 norm.
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle as O  # noqa: E402

SETTINGS = settings(max_examples=25, deadline=None, derandomize=True)
axis = st.integers(min_value=2, max_value=12)
seeds = st.integers(min_value=0, max_value=2**31 - 1)


@st.composite
def grids(draw, dims=(2, 3)):
    dim = draw(st.sampled_from(dims))
    n = tuple(draw(axis) if dim == 2 else draw(st.integers(2, 6)) for _ in range(dim))
    L = tuple(draw(st.floats(0.3, 3.0)) for _ in range(dim))
    return O.Grid(n, L)


def fields(g, seed):
    rng = np.random.default_rng(seed)
    m = rng.uniform(-1, 1, (g.dim,) + g.shape)
    r = rng.uniform(0.05, 0.5, g.shape)
    return rng, m, r


@SETTINGS
@given(grids(), seeds)
def test_transform_round_trip_and_parseval(g, seed):
    rng = np.random.default_rng(seed)
    f = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
    F = O.fftn(g, f, -1)
    back = O.fftn(g, F, +1)   # the inverse carries the 1/n
    assert np.allclose(back, f, atol=1e-12)
    assert np.isclose((abs(F) ** 2).sum(), g.npts * (abs(f) ** 2).sum(), rtol=1e-12)


@SETTINGS
@given(grids(), seeds)
def test_operator_symmetric_psd_and_blind_to_the_null_space(g, seed):
    rng, m, r = fields(g, seed)
    u, v = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    Au, Av = O.apply_A(g, m, r, u), O.apply_A(g, m, r, v)
    scale = np.abs(Au).max() * np.abs(v).max() * g.npts
    assert abs((v * Au).sum() - (u * Av).sum()) <= 1e-12 * scale
    assert (u * Au).sum() >= -1e-12 * scale
    assert np.allclose(O.apply_A(g, m, r, O.project(g, u)), Au, atol=1e-11 * np.abs(Au).max())


@SETTINGS
@given(grids(), seeds)
def test_projection_idempotent_and_orthogonal(g, seed):
    f = np.random.default_rng(seed).standard_normal(g.shape)
    P = O.project(g, f)
    assert np.allclose(O.project(g, P), P, atol=1e-13)
    assert abs((P * (f - P)).sum()) <= 1e-12 * (f * f).sum()
    assert abs(P.sum()) <= 1e-11 * np.abs(f).sum()   # the constant mode is always removed


@SETTINGS
@given(st.integers(2, 3), seeds, st.floats(0.05, 3.0), st.floats(1e-4, 0.5))
def test_relaxation_keeps_direction_and_never_grows(dim, seed, gamma, dt):
    m = np.random.default_rng(seed).uniform(-1, 1, (dim, 64))
    out = O.relaxation(m, gamma, dt)
    nm, no = np.linalg.norm(m, axis=0), np.linalg.norm(out, axis=0)
    assert np.all(no <= nm * (1 + 1e-14))
    alive = no > 0
    cosang = (m * out).sum(0)[alive] / (nm[alive] * no[alive])
    assert np.allclose(cosang, 1.0, atol=1e-12)


@SETTINGS
@given(st.integers(2, 3), seeds, st.floats(0.0, 5.0), st.floats(1e-4, 0.2))
def test_activation_changes_only_the_part_along_the_gradient(dim, seed, c, dt):
    rng = np.random.default_rng(seed)
    m = rng.uniform(-1, 1, (dim, 64))
    gp = rng.uniform(-1, 1, (dim, 64))
    out = O.activation(m, gp, c, dt)
    g2 = (gp * gp).sum(0)
    along_in, along_out = (m * gp).sum(0), (out * gp).sum(0)
    perp_in = m - along_in / g2 * gp
    perp_out = out - along_out / g2 * gp
    assert np.allclose(perp_out, perp_in, atol=1e-12)
    assert np.all(np.abs(along_out) >= np.abs(along_in) * (1 - 1e-14))
    assert np.all(np.sign(along_out) == np.sign(along_in))


@SETTINGS
@given(grids(), seeds, st.floats(0.0, 0.3), st.floats(1e-4, 0.1))
def test_diffusion_keeps_means_and_never_grows_the_norm(g, seed, D, dt):
    _, m, _ = fields(g, seed)
    out = O.diffusion(g, m, D, dt)
    for c in range(g.dim):
        assert np.isclose(out[c].mean(), m[c].mean(), atol=1e-13)
        assert np.linalg.norm(out[c]) <= np.linalg.norm(m[c]) * (1 + 1e-13)


@SETTINGS
@given(grids(dims=(2,)), seeds, st.floats(0.5, 2.0), st.floats(0.1, 1.0), st.floats(0.3, 3.0))
def test_energy_scales_term_by_term(g, seed, gamma, D, lam):
    """With c = 0 the energy of Section 2.5 has two terms of fixed degree:
    E(lam m) = lam^2 E_diff(m) + lam^(2 gamma) E_relax(m). E_diff is the energy
    with the relaxation term scaled out, E_relax the one with D = 0."""
    _, m, r = fields(g, seed)
    p = np.zeros(g.shape)
    full = O.Params(c=0.0, D=D, gamma=gamma, dt=1e-3)
    no_diff = O.Params(c=0.0, D=0.0, gamma=gamma, dt=1e-3)
    E_relax = O.energy(g, no_diff, r, m, p)
    E_diff = O.energy(g, full, r, m, p) - E_relax
    got = O.energy(g, full, r, lam * m, p)
    want = lam ** 2 * E_diff + lam ** (2 * gamma) * E_relax
    assert np.isclose(got, want, rtol=1e-11)
    assert E_diff >= 0 and E_relax > 0


@SETTINGS
@given(grids(), seeds, st.floats(1e-4, 0.3), st.floats(0.3, 3.0))
def test_gamma0_energy_is_the_log_limit_and_relaxation_never_raises_it(g, seed, dt, lam):
    """Reading R21: at gamma = 0 the relaxation term of the energy is
    h sum ln|m|, the gamma -> 0 limit of h sum (|m|^(2 gamma) - 1)/(2 gamma).
    (i) It is that limit: E_gamma(m) - |Omega|/(2 gamma) -> E_0(m), with an
    O(gamma) gap. (ii) Scaling m by lam adds |Omega| ln lam. (iii) Pure
    relaxation at gamma = 0 (the flow of that term) never raises it, and a
    point it extinguishes makes it -inf."""
    _, m, r = fields(g, seed)
    p = np.zeros(g.shape)
    vol = float(np.prod(g.L))

    def E(gamma, mm):
        return O.energy(g, O.Params(c=0.0, D=0.0, gamma=gamma, dt=dt), r, mm, p)

    E0 = E(0.0, m)
    assert np.isfinite(E0)
    h = vol / g.npts
    assert np.isclose(E0, h * np.log(np.linalg.norm(m, axis=0)).sum(), rtol=1e-12, atol=1e-12)
    for gam in (1e-5, 1e-6):
        gap = E(gam, m) - vol / (2 * gam) - E0
        assert abs(gap) < 50 * gam * (vol + abs(E0) + 1)
    assert np.isclose(E(0.0, lam * m), E0 + vol * np.log(lam), rtol=1e-11, atol=1e-11)
    mk = m
    for _ in range(4):
        mn = O.relaxation(mk, 0.0, dt)
        before, after = E(0.0, mk), E(0.0, mn)
        assert after <= before or (np.isneginf(after) and np.isneginf(before))
        if np.any(np.linalg.norm(mn, axis=0) == 0):
            assert np.isneginf(after)
        mk = mn


@SETTINGS
@given(grids(), seeds)
def test_preconditioner_is_symmetric_positive_on_the_range(g, seed):
    """M^-1 of reading R3 (both options) is symmetric, positive on the
    complement of the null space, and zero on the null space."""
    rng, m, r = fields(g, seed)
    u = O.project(g, rng.standard_normal(g.shape))
    v = O.project(g, rng.standard_normal(g.shape))
    for kb in (O.kappa_default(g, m, r), O.kbar_default(g, m, r)):
        Mu, Mv = O.precond(g, kb, u), O.precond(g, kb, v)
        scale = np.abs(Mu).max() * np.abs(v).max() * g.npts
        assert abs((v * Mu).sum() - (u * Mv).sum()) <= 1e-12 * scale
        if g.npts > np.prod([2 if N % 2 == 0 else 1 for N in g.n]):   # the range is not empty
            assert (u * Mu).sum() > 0
        null = u - O.project(g, u) + (rng.standard_normal() * np.ones(g.shape))
        assert np.abs(O.precond(g, kb, null)).max() <= 1e-12 * (1 + np.abs(null).max())


@settings(max_examples=20, deadline=None, derandomize=True)
@given(grids(), seeds, st.floats(0.5, 1.5))
def test_step_keeps_p_in_the_range_and_repeats_exactly(g, seed, gamma):
    """Reading R2: after a step p has no null-space component. The step is a
    deterministic function of its inputs, and the energy of its state is
    finite and non-negative."""
    rng, m, r = fields(g, seed)
    S = rng.standard_normal(g.shape)
    prm = O.Params(c=2.0, D=0.05, gamma=gamma, dt=1e-3, cg_rtol=1e-10)
    m1, p1, st1 = O.step(g, prm, r, S, m, np.zeros(g.shape))
    m2, p2, st2 = O.step(g, prm, r, S, m, np.zeros(g.shape))
    assert st1.rc in (O.OK, O.ENOCONV)
    assert np.allclose(O.project(g, p1), p1, atol=1e-12 * (1 + np.abs(p1).max()))
    assert np.array_equal(m1, m2) and np.array_equal(p1, p2)
    E = O.energy(g, prm, r, m, p1)
    assert np.isfinite(E) and E >= 0


@settings(max_examples=12, deadline=None, derandomize=True)
@given(st.tuples(st.integers(3, 8), st.integers(3, 8)), seeds)
def test_adjoint_directional_derivative_on_random_grids(n, seed):
    """<dL/dm0, dm> equals the central difference of L = <w, m(T)> along a
    random direction dm, on small odd and even grids (gamma = 1 keeps the
    relaxation smooth; m stays away from 0)."""
    g = O.Grid(n, (1.0, 0.8))
    rng = np.random.default_rng(seed)
    m0 = rng.uniform(0.3, 1.0, (2,) + g.shape)
    r = rng.uniform(0.05, 0.3, g.shape)
    S = rng.standard_normal(g.shape)
    prm = O.Params(c=2.0, D=0.1, gamma=1.0, dt=2e-3, cg_rtol=1e-14, cg_maxit=2000)
    w = rng.standard_normal(m0.shape)
    dm = rng.standard_normal(m0.shape)
    adj = O.adjoint(g, prm, r, S, m0, np.zeros(g.shape), 2, w)

    def L(h):
        m, p = m0 + h * dm, np.zeros(g.shape)
        for _ in range(2):
            m, p, _ = O.step(g, prm, r, S, m, p)
        return float((w * m).sum())

    h = 1e-6
    fd = (L(h) - L(-h)) / (2 * h)
    got = float((adj["dm0"] * dm).sum())
    assert np.isfinite(got) and abs(got - fd) <= 1e-6 * (abs(fd) + np.abs(adj["dm0"]).sum())


@settings(max_examples=12, deadline=None, derandomize=True)
@given(grids(dims=(2,)), seeds, st.floats(0.5, 1.5), st.sampled_from([0.0, 1e-3, 10.0]),
       st.booleans())
def test_run_reports_consistent_results(g, seed, gamma, eps, stop_on_energy):
    """Algorithm 1's loop (Section 2.5): a stop reason from the list, at most
    max_steps bodies, one energy and one Delta m per completed body, finite
    values, and the energy rule naming the step before the one that saw it."""
    rng, m, r = fields(g, seed)
    S = rng.standard_normal(g.shape)
    prm = O.Params(c=2.0, D=0.05, gamma=gamma, dt=1e-3, cg_rtol=1e-10)
    res = O.run(g, prm, r, S, m, max_steps=5, eps=eps, stop_on_energy=stop_on_energy)
    assert res.reason in (0, 1, 2) and 1 <= res.steps <= 5
    assert len(res.energies) == len(res.delta_ms) == res.steps
    assert all(np.isfinite(res.energies)) and all(np.isfinite(res.delta_ms))
    if res.reason == 0:
        assert res.steps == 5
    if res.reason == 1:
        assert eps > 0 and res.delta_ms[-1] <= eps
    if res.reason == 2:
        assert stop_on_energy and res.energies[-1] >= res.energies[-2]
        assert res.energy_step == res.steps - 2


@SETTINGS
@given(grids(), seeds)
def test_gradient_is_exact_below_the_nyquist_index(g, seed):
    """Section 2.3.3's Fourier variables: for a trigonometric polynomial whose
    modes all lie strictly below N/2 along every axis, the spectral gradient
    equals the exact derivative, on odd and even grids alike."""
    rng = np.random.default_rng(seed)
    X = np.meshgrid(*[np.arange(N) * (L / N) for N, L in zip(g.n, g.L)][::-1], indexing="ij")[::-1]
    f = np.zeros(g.shape)
    df = np.zeros((g.dim,) + g.shape)
    for _ in range(3):
        k = [int(rng.integers(-((N - 1) // 2), (N - 1) // 2 + 1)) for N in g.n]
        a, b = rng.standard_normal(2)
        arg = sum(2 * np.pi * kk * Xa / L for kk, Xa, L in zip(k, X, g.L))
        f += a * np.cos(arg) + b * np.sin(arg)
        for ax in range(g.dim):
            w = 2 * np.pi * k[ax] / g.L[ax]
            df[ax] += w * (-a * np.sin(arg) + b * np.cos(arg))
    assert np.allclose(O.gradient(g, f), df, atol=1e-11 * (1 + np.abs(df).max()))


@settings(max_examples=10, deadline=None, derandomize=True)
@given(grids(), seeds, st.integers(1, 4))
def test_run_without_stops_equals_repeated_steps(g, seed, k):
    """Algorithm 1's loop with both rules off is k loop bodies: the state it
    returns is bit-identical to stepping by hand."""
    rng, m, r = fields(g, seed)
    S = rng.standard_normal(g.shape)
    prm = O.Params(c=2.0, D=0.05, gamma=0.75, dt=1e-3, cg_rtol=1e-10)
    res = O.run(g, prm, r, S, m, max_steps=k, eps=0.0, stop_on_energy=False)
    mm, pp = m.copy(), np.zeros(g.shape)
    for _ in range(k):
        mm, pp, _ = O.step(g, prm, r, S, mm, pp)
    assert res.reason == 0 and res.steps == k
    assert np.array_equal(res.m, mm) and np.array_equal(res.p, pp)


@settings(max_examples=8, deadline=None, derandomize=True)
@given(st.tuples(st.integers(3, 5), st.integers(3, 5), st.integers(3, 5)), seeds)
def test_adjoint_directional_derivative_on_random_3d_grids(n, seed):
    """As the 2D case: <dL/dm0, dm> against a central difference along a random
    dm, on small 3D grids, and <dL/dS, dS> along a random source direction."""
    g = O.Grid(n, (1.0, 0.7, 1.3))
    rng = np.random.default_rng(seed)
    m0 = rng.uniform(0.3, 1.0, (3,) + g.shape)
    r = rng.uniform(0.05, 0.3, g.shape)
    S = rng.standard_normal(g.shape)
    prm = O.Params(c=2.0, D=0.1, gamma=1.0, dt=2e-3, cg_rtol=1e-14, cg_maxit=2000)
    w = rng.standard_normal(m0.shape)
    dm, dS = rng.standard_normal(m0.shape), rng.standard_normal(g.shape)
    adj = O.adjoint(g, prm, r, S, m0, np.zeros(g.shape), 2, w)

    def L(hm, hs):
        m, p = m0 + hm * dm, np.zeros(g.shape)
        for _ in range(2):
            m, p, _ = O.step(g, prm, r, S + hs * dS, m, p)
        return float((w * m).sum())

    h = 1e-6
    fd_m = (L(h, 0) - L(-h, 0)) / (2 * h)
    fd_s = (L(0, h) - L(0, -h)) / (2 * h)
    got_m = float((adj["dm0"] * dm).sum())
    got_s = float((adj["dS"] * dS).sum())
    assert abs(got_m - fd_m) <= 1e-6 * (abs(fd_m) + np.abs(adj["dm0"]).sum())
    assert abs(got_s - fd_s) <= 1e-6 * (abs(fd_s) + np.abs(adj["dS"]).sum())
