"""GPU adjoint (hc_adjoint) against the oracle's discrete adjoint, against
central finite differences of the GPU's own forward map (64^2, the size the
gradients are checked at), checkpoint invariance, and the torch.autograd
wrapper."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import hc, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu


def problem(n=64):
    w = W.source_sink_2d(n, steps=4, gamma=0.75)
    # a gentler step so a few steps keep |grad p| moderate and gradients smooth
    w.c, w.dt = 10.0, 1e-3
    return w


def make(hc, w, precision="fp64", rtol=1e-13):
    s = hc.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision=precision,
                  cg_rtol=rtol, cg_maxit=5000)
    s.set_r(w.r)
    s.set_source(w.S)
    s.set_m(w.m0)
    return s


def test_adjoint_matches_oracle_adjoint_fp64(hc):
    w = problem(64)
    g = O.Grid(w.n, w.L)
    rng = np.random.default_rng(4)
    lam = rng.standard_normal((2,) + w.shape)
    prm = O.Params(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-13, cg_maxit=5000)
    ref = O.adjoint(g, prm, w.r, w.S, w.m0, np.zeros(w.shape), 4, lam)
    with make(hc, w) as s:
        got = s.adjoint(4, lam, every=2)
    assert np.isclose(got["dc2"], ref["dc2"], rtol=1e-8)
    assert np.isclose(got["dD2"], ref["dD2"], rtol=1e-8)
    for k in ("dr", "dS", "dm0"):
        assert rel_l2(got[k], ref[k]) < 1e-8, k


def special_problem(case):
    """The regimes where the adjoint's pointwise Jacobians switch branch:
    conductivity exactly 0 and conductivity that dies out in one step (gamma
    < 1), m = 0 with gamma > 1, activation exponents past the phi_1' series
    range, and no activation at all (c = 0)."""
    w = problem(64)
    if case in ("zero_and_extinct", "zero_gamma_above_one"):
        w.gamma = 0.5 if case == "zero_and_extinct" else 1.5
        for j, i in [(5, 9), (40, 13), (63, 0)]:
            w.m0[:, j, i] = 0.0
        if case == "zero_and_extinct":
            for j, i in [(20, 30), (0, 63)]:
                w.m0[:, j, i] = (0.3 * w.dt, -0.2 * w.dt)
    elif case == "large_exponent":
        g = O.Grid(w.n, w.L)
        prm = O.Params(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-13, cg_maxit=5000)
        _, p1, _ = O.step(g, prm, w.r, w.S, w.m0.copy(), np.zeros(w.shape))
        g2 = (O.gradient(g, p1) ** 2).sum(0)
        w.c = float(np.sqrt(2.0 / (w.dt * g2.max())))   # largest c^2 dt |grad p|^2 about 2
    elif case == "no_activation":
        w.c = 0.0
    return w


@pytest.mark.parametrize("case", ["zero_and_extinct", "zero_gamma_above_one", "large_exponent",
                                  "no_activation"])
def test_adjoint_special_regimes_match_oracle(hc, case):
    w = special_problem(case)
    g = O.Grid(w.n, w.L)
    lam = np.random.default_rng(9).standard_normal((2,) + w.shape)
    prm = O.Params(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-13, cg_maxit=5000)
    ref = O.adjoint(g, prm, w.r, w.S, w.m0, np.zeros(w.shape), 3, lam)
    with make(hc, w) as s:
        got = s.adjoint(3, lam, every=2)
    assert np.isclose(got["dc2"], ref["dc2"], rtol=1e-8), (got["dc2"], ref["dc2"])
    assert np.isclose(got["dD2"], ref["dD2"], rtol=1e-8)
    for k in ("dr", "dS", "dm0"):
        assert rel_l2(got[k], ref[k]) < 1e-8, k


def test_adjoint_matches_central_differences_on_gpu(hc):
    """Finite differences of the GPU forward itself at 64^2: relative error
    <= 1e-4 for dL/dc^2, dL/dD^2 and sampled entries of dL/dr, dL/dS, dL/dm0."""
    w = problem(64)
    rng = np.random.default_rng(5)
    lam = rng.standard_normal((2,) + w.shape)
    nsteps = 3

    def L_of(c=None, D=None, r=None, S=None, m0=None):
        c = w.c if c is None else c
        D = w.D if D is None else D
        with hc.Solver(w.n, w.L, c=c, D=D, gamma=w.gamma, dt=w.dt, precision="fp64",
                       cg_rtol=1e-14, cg_maxit=5000) as s:
            s.set_r(w.r if r is None else r)
            s.set_source(w.S if S is None else S)
            s.set_m(w.m0 if m0 is None else m0)
            s.step(nsteps)
            return float((lam * s.get_m()).sum())

    with make(hc, w, rtol=1e-14) as s:
        adj = s.adjoint(nsteps, lam, every=2)
    c2, D2 = w.c ** 2, w.D ** 2
    h = 1e-4 * c2
    fd = (L_of(c=np.sqrt(c2 + h)) - L_of(c=np.sqrt(c2 - h))) / (2 * h)
    assert abs(adj["dc2"] - fd) <= 1e-4 * abs(fd)
    h = 1e-3 * D2
    fd = (L_of(D=np.sqrt(D2 + h)) - L_of(D=np.sqrt(D2 - h))) / (2 * h)
    assert abs(adj["dD2"] - fd) <= 1e-4 * abs(fd)
    for (j, i) in [(10, 20), (33, 47)]:
        for key, field in (("dr", w.r), ("dS", w.S)):
            hp, hm = field.copy(), field.copy()
            hp[j, i] += 1e-5
            hm[j, i] -= 1e-5
            fd = (L_of(**{key[1:]: hp}) - L_of(**{key[1:]: hm})) / 2e-5
            assert abs(adj[key][j, i] - fd) <= 1e-4 * np.abs(adj[key]).max(), key
        mp, mm = w.m0.copy(), w.m0.copy()
        mp[1, j, i] += 1e-6
        mm[1, j, i] -= 1e-6
        fd = (L_of(m0=mp) - L_of(m0=mm)) / 2e-6
        assert abs(adj["dm0"][1, j, i] - fd) <= 1e-4 * np.abs(adj["dm0"]).max()


def test_checkpoint_spacing_does_not_change_the_gradient(hc):
    w = problem(64)
    lam = np.random.default_rng(6).standard_normal((2,) + w.shape)
    outs = []
    for every in (1, 2, 5):
        with make(hc, w) as s:
            outs.append(s.adjoint(5, lam, every=every))
    for o in outs[1:]:
        assert o["dc2"] == outs[0]["dc2"] and o["dD2"] == outs[0]["dD2"]
        for k in ("dr", "dS", "dm0"):
            assert np.array_equal(o[k], outs[0][k])


def test_adjoint_leaves_the_forward_state(hc):
    w = problem(64)
    lam = np.random.default_rng(7).standard_normal((2,) + w.shape)
    with make(hc, w) as s:
        s.step(3)
        m_ref, p_ref = s.get_m(), s.get_p()
    with make(hc, w) as s:
        s.adjoint(3, lam, every=2)
        assert np.array_equal(s.get_m(), m_ref)
        assert np.array_equal(s.get_p(), p_ref)


def test_refined_adjoint_close_to_oracle(hc):
    """FP32 forward with FP64 refinement: gradients to FP32 accuracy."""
    w = problem(128)
    g = O.Grid(w.n, w.L)
    lam = np.random.default_rng(8).standard_normal((2,) + w.shape)
    prm = O.Params(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-12, cg_maxit=5000)
    ref = O.adjoint(g, prm, w.r, w.S, w.m0, np.zeros(w.shape), 3, lam)
    with make(hc, w, "fp32_refined", rtol=1e-9) as s:
        got = s.adjoint(3, lam, every=2)
    assert np.isclose(got["dc2"], ref["dc2"], rtol=1e-3)
    assert np.isclose(got["dD2"], ref["dD2"], rtol=1e-3)
    for k in ("dr", "dS", "dm0"):
        assert rel_l2(got[k], ref[k]) < 1e-3, k


def test_refined_adjoint_matches_fp64_gpu_adjoint_256(hc):
    """The refined path's gradients (FP32 forward states and reverse passes,
    FP64-certified pressure solves) against the plain FP64 GPU adjoint at 256^2
    over 10 steps with a checkpoint every 5, the shape of the 1024^2 adjoint
    configuration at a size both paths run in seconds.  Bound 2e-3 relative:
    the FP32 states carry u32 ~ 6e-8, which the chain rule amplifies through the
    steps by the loss's sensitivity (the 3-step oracle comparison above holds
    1e-3)."""
    w = problem(256)
    lam = np.random.default_rng(9).standard_normal((2,) + w.shape)
    with make(hc, w, "fp64", rtol=1e-12) as s:
        ref = s.adjoint(10, lam, every=5)
    with make(hc, w, "fp32_refined", rtol=1e-9) as s:
        got = s.adjoint(10, lam, every=5)
    assert np.isclose(got["dc2"], ref["dc2"], rtol=2e-3), (got["dc2"], ref["dc2"])
    assert np.isclose(got["dD2"], ref["dD2"], rtol=2e-3), (got["dD2"], ref["dD2"])
    for k in ("dr", "dS", "dm0"):
        assert rel_l2(got[k], ref[k]) < 2e-3, k


def test_adjoint_at_1024_against_differences_and_fp64(hc):
    """The 1024^2 adjoint configuration (smooth r, source/sink S, c = 25,
    D = 0.02, gamma = 0.75, dt = 5e-4) at its full grid, over 4 steps with a
    checkpoint every 2: the plain FP64 GPU adjoint against central differences
    of the FP64 forward (rtol 1e-13) for dL/dc^2, dL/dD^2 and the directional
    derivative of L along a smooth perturbation of r, within 1e-4; and the
    refined path's gradients against that FP64 adjoint within 2e-3 (the bound
    of the 256^2 comparison above)."""
    w = W.source_sink_2d(1024, steps=4, gamma=0.75)
    nsteps = 4
    lam = np.random.default_rng(11).standard_normal((2,) + w.shape)
    dr = 0.01 * W.smooth_field(w.n, 3, 8, w.L)

    def L_of(c2=None, D2=None, r=None):
        c = w.c if c2 is None else np.sqrt(c2)
        D = w.D if D2 is None else np.sqrt(D2)
        with hc.Solver(w.n, w.L, c=c, D=D, gamma=w.gamma, dt=w.dt, precision="fp64",
                       cg_rtol=1e-13, cg_maxit=5000) as s:
            s.set_r(w.r if r is None else r)
            s.set_source(w.S)
            s.set_m(w.m0)
            s.step(nsteps)
            return float((lam * s.get_m()).sum())

    with make(hc, w, "fp64", rtol=1e-13) as s:
        ref = s.adjoint(nsteps, lam, every=2)
    c2, D2 = w.c ** 2, w.D ** 2
    h = 1e-4 * c2
    fd = (L_of(c2=c2 + h) - L_of(c2=c2 - h)) / (2 * h)
    assert abs(ref["dc2"] - fd) <= 1e-4 * abs(fd), (ref["dc2"], fd)
    h = 1e-3 * D2
    fd = (L_of(D2=D2 + h) - L_of(D2=D2 - h)) / (2 * h)
    assert abs(ref["dD2"] - fd) <= 1e-4 * abs(fd), (ref["dD2"], fd)
    h = 1e-2
    fd = (L_of(r=w.r + h * dr) - L_of(r=w.r - h * dr)) / (2 * h)
    dd = float((ref["dr"] * dr).sum())
    assert abs(dd - fd) <= 1e-4 * abs(fd), (dd, fd)
    with make(hc, w, "fp32_refined", rtol=1e-9) as s:
        got = s.adjoint(nsteps, lam, every=2)
    assert np.isclose(got["dc2"], ref["dc2"], rtol=2e-3), (got["dc2"], ref["dc2"])
    assert np.isclose(got["dD2"], ref["dD2"], rtol=2e-3), (got["dD2"], ref["dD2"])
    for k in ("dr", "dS", "dm0"):
        assert rel_l2(got[k], ref[k]) < 2e-3, k


def test_autograd_function(hc):
    import torch
    w = problem(64)
    with make(hc, w) as s:
        c2 = torch.tensor(w.c ** 2, dtype=torch.float64, requires_grad=True)
        D2 = torch.tensor(w.D ** 2, dtype=torch.float64, requires_grad=True)
        r = torch.from_numpy(w.r.copy()).requires_grad_()
        S = torch.from_numpy(w.S.copy()).requires_grad_()
        m0 = torch.from_numpy(w.m0.copy()).requires_grad_()
        target = torch.from_numpy(np.full((2,) + w.shape, 0.2))
        mT = hc.hucai_steps(s, 2, 1, c2, D2, r, S, m0)
        loss = ((mT - target) ** 2).sum()
        loss.backward()
        lam = 2 * (mT.detach().numpy() - 0.2)
        s.set_params(c=w.c, D=w.D)
        s.set_r(w.r); s.set_source(w.S); s.set_m(w.m0); s.set_p(np.zeros(w.shape))
        ref = s.adjoint(2, lam, every=1)
    assert np.isclose(c2.grad.item(), ref["dc2"], rtol=1e-12)
    assert np.allclose(m0.grad.numpy(), ref["dm0"], rtol=1e-12, atol=0)
    assert np.allclose(r.grad.numpy(), ref["dr"], rtol=1e-12, atol=0)
