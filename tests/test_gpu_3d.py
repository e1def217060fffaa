"""GPU parity of the 3D step (d = 3) against the FP64 oracle, through the C
ABI: the 3D transform (x rows, y and z passes), the spectral gradient, the
pressure operator of eq. (p_discrete), the split step of Section 2.3, whole
steps of Algorithm 1 in both precisions, and, at the 256^3 source/sink
workload, the FP64 pressure residual measured with the oracle's own operator
plus the split step recomputed by the oracle.

Shapes span several tiles in every pass, unequal axes and lengths, the
minimum transform length 8 and long thin grids."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import hc, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(33)
TOL = {"fp64": 1e-12, "fp32_refined": 2e-6, "fp32_refined_df": 2e-6}
SHAPES3 = [(8, 8, 8), (16, 8, 32), (32, 64, 16), (8, 128, 8), (128, 8, 16), (64, 64, 64),
           (1024, 8, 16), (8, 1024, 8), (16, 8, 1024)]   # the last three: the longest axes


def packed3(F: np.ndarray) -> np.ndarray:
    """Packed half-spectrum of a full 3D spectrum F[kz, ky, kx]: kx < nx/2,
    with F[..., 0] + i F[..., nx/2] in the kx = 0 slot."""
    H = F.shape[-1] // 2
    P = F[..., :H].copy()
    P[..., 0] = F[..., 0] + 1j * F[..., H]
    return P


def solver(hc, n, L=None, precision="fp64", **kw):
    args = dict(c=10.0, D=0.05, gamma=0.75, dt=1e-3)
    args.update(kw)
    return hc.Solver(n, L, precision=precision, **args)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
@pytest.mark.parametrize("n", SHAPES3)
def test_spectrum_3d_matches_oracle_transform(hc, precision, n):
    g = O.Grid(n)
    f = RNG.standard_normal(g.shape)
    with solver(hc, n, precision=precision) as s:
        P = s.spectrum(f)
    assert P.shape == (n[2], n[1], n[0] // 2)
    assert rel_l2(P, packed3(O.fftn(g, f, -1))) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined", "fp32_refined_df"])
@pytest.mark.parametrize("n,L", [((16, 8, 32), (1.0, 0.5, 2.0)), ((8, 8, 8), (1.0, 1.0, 1.0)),
                                 ((64, 32, 16), (2.0, 1.0, 1.0))])
def test_gradient_3d_matches_oracle(hc, precision, n, L):
    g = O.Grid(n, L)
    p = RNG.standard_normal(g.shape)
    with solver(hc, n, L, precision=precision) as s:
        s.set_p(p)
        grad = s.gradient()
        p_back = s.get_p()
    pp = O.project(g, p)
    assert rel_l2(p_back, pp) < (1e-13 if precision != "fp32_refined_df" else 1e-12)
    assert rel_l2(grad, O.gradient(g, pp)) < TOL[precision] * 2


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
@pytest.mark.parametrize("n,L", [((16, 8, 32), (1.0, 0.5, 2.0)), ((32, 32, 32), (1.0, 1.0, 1.0)),
                                 ((8, 64, 16), (1.0, 1.0, 0.5)), ((1024, 8, 8), (2.0, 1.0, 1.0)),
                                 ((8, 8, 1024), (1.0, 1.0, 1.0))])
def test_operator_3d_matches_oracle(hc, precision, n, L):
    g = O.Grid(n, L)
    m = RNG.uniform(-0.5, 0.5, (3,) + g.shape)
    r = RNG.uniform(0.05, 0.15, g.shape)
    f = RNG.standard_normal(g.shape)
    with solver(hc, n, L, precision=precision) as s:
        s.set_m(m)
        s.set_r(r)
        Af = s.apply_operator(f)
    ref = O.apply_A(g, m, r, O.project(g, f))
    assert rel_l2(Af, ref) < TOL[precision] * 5


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
@pytest.mark.parametrize("gamma", [0.25, 0.5, 0.75, 0.999, 1.0, 1.001, 1.5])
def test_split_step_3d_matches_oracle(hc, precision, gamma):
    """Step 2 of Algorithm 1 with p given, including |m| = 0 planes and
    points that relaxation extinguishes; the GPU applies the diffusion as
    three 1D heat operators, the oracle as one 3D multiplier."""
    n, L = (32, 16, 8), (1.0, 0.5, 0.25)
    g = O.Grid(n, L)
    Z, Y, X = np.meshgrid(np.arange(n[2]) * L[2] / n[2], np.arange(n[1]) * L[1] / n[1],
                          np.arange(n[0]) * L[0] / n[0], indexing="ij")
    p = (np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y / L[1])
         + 0.2 * np.cos(2 * np.pi * Z / L[2]) + 0.003 * RNG.standard_normal(g.shape))
    m = RNG.uniform(-0.5, 0.5, (3,) + g.shape)
    m[:, 2, :, :] = 0.0
    m[:, 5, 3, :] = 1e-4
    c, D, dt = 1.0, 0.05, 2e-3
    with solver(hc, n, L, precision=precision, c=c, D=D, gamma=gamma, dt=dt) as s:
        s.set_p(p)
        s.set_m(m)
        s.split_step()
        got = s.get_m()
    pp = O.project(g, p)
    mm = m if precision == "fp64" else m.astype(np.float32).astype(np.float64)
    gp = O.gradient(g, pp)
    ref = O.diffusion(g, O.relaxation(O.activation(mm, gp, c, dt), gamma, dt), D, dt)
    assert (c * c * dt * (gp ** 2).sum(0)).max() < 10
    assert rel_l2(got, ref) < (1e-12 if precision == "fp64" else 2e-6)


def _problem(n, L, seed=0):
    g = O.Grid(n, L)
    r = RNG.uniform(0.05, 0.15, g.shape)
    S = W.minus_mean(W.gaussian(n, (0.3, 0.5, 0.5), 0.1, L) - W.gaussian(n, (0.7, 0.5, 0.5), 0.1, L))
    m0 = W.uniform_m(g.shape, 3, 0.0, 0.5, seed)
    return g, r, S, m0


@pytest.mark.parametrize("use_graph", [True, False])
def test_steps_3d_fp64_match_oracle_per_step(hc, use_graph):
    """FP64 plain: relative L2 of m and p within 1e-10 of the oracle after
    every step."""
    n, L = (16, 32, 8), (1.0, 2.0, 0.5)
    g, r, S, m0 = _problem(n, L)
    prm = O.Params(c=3.0, D=0.05, gamma=0.75, dt=1e-3, cg_rtol=1e-12, cg_maxit=2000)
    m_ref, p_ref = m0.copy(), np.zeros(g.shape)
    with solver(hc, n, L, "fp64", c=prm.c, D=prm.D, gamma=prm.gamma, dt=prm.dt,
                cg_rtol=prm.cg_rtol, cg_maxit=prm.cg_maxit, use_graph=use_graph) as s:
        s.set_r(r)
        s.set_source(S)
        s.set_m(m0)
        for k in range(4):
            st = s.step(1)
            m_ref, p_ref, ost = O.step(g, prm, r, S, m_ref, p_ref)
            assert st.status == hc.HC_OK
            assert rel_l2(s.get_m(), m_ref) < 1e-10, k
            assert rel_l2(s.get_p(), p_ref) < 1e-10, k


@pytest.mark.parametrize("precision", ["fp32_refined", "fp32_refined_df"])
def test_steps_3d_refined_match_oracle(hc, precision):
    """FP32 + FP64 refinement on the 3D source/sink problem at 32^3: the
    pressure residual measured with the oracle's FP64 operator stays at or
    below 1e-8, and m stays within 1e-5 of the oracle over 30 steps.  The
    refined path stores m and r in FP32, so the residual is measured with
    those stored coefficients."""
    w = W.source_sink_3d(32)
    g = O.Grid(w.n, w.L)
    prm = O.Params(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-12, cg_maxit=3000)
    m_ref, p_ref = w.m0.copy(), np.zeros(g.shape)
    with solver(hc, w.n, w.L, precision, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-8) as s:
        s.set_r(w.r)
        s.set_source(w.S)
        s.set_m(w.m0)
        m_prev = s.get_m()
        r32 = w.r.astype(np.float32).astype(np.float64)
        for k in range(30):
            st = s.step(1)
            assert st.status == hc.HC_OK and st.refine_sweeps >= 1
            p = s.get_p()
            res = O.project(g, w.S) - O.apply_A(g, m_prev, r32, p)
            assert np.linalg.norm(res) <= 1e-8 * np.linalg.norm(O.project(g, w.S)), k
            m_prev = s.get_m()
            m_ref, p_ref, _ = O.step(g, prm, w.r, w.S, m_ref, p_ref)
        assert rel_l2(m_prev, m_ref) < 1e-5
        assert rel_l2(p, p_ref) < 1e-6


def test_double_float_mid_residual_3d(hc):
    """3D fp32_refined: the residual after the FP32 first sweep is evaluated in
    double-float; every step still ends on an FP64 residual (checked with the
    oracle's operator), one fewer per step than with fp64_mid_residual, and
    the graph counts the mid-step block's kernels."""
    w = W.source_sink_3d(32)
    g = O.Grid(w.n, w.L)
    b = O.project(g, w.S)
    r32 = w.r.astype(np.float32).astype(np.float64)
    outs, extra = [], []
    for fp64_mid in (False, True):
        with solver(hc, w.n, w.L, "fp32_refined", c=w.c, D=w.D, gamma=w.gamma, dt=w.dt,
                    cg_rtol=1e-8, fp64_mid_residual=fp64_mid) as s:
            s.set_r(w.r)
            s.set_source(w.S)
            s.set_m(w.m0)
            for k in range(5):
                m_prev = s.get_m()
                before = s.launch_count()
                st = s.step(1)
                launched = s.launch_count() - before
                assert st.status == hc.HC_OK and st.first_sweep_fp32 == 1
                assert st.mid_residual_df == (0 if fp64_mid else 1)
                # each sweep after the FP32 one starts from an FP64 residual, and one
                # more certifies; the double-float residual starts the second sweep
                # (or, already below the target, replaces it)
                want = st.refine_sweeps if fp64_mid else max(1, st.refine_sweeps - 1)
                assert st.refine_residuals == want, (k, st)
                res = b - O.apply_A(g, m_prev, r32, s.get_p())
                assert np.linalg.norm(res) <= 1.2e-8 * np.linalg.norm(b), k
                # fixed nodes, 6 per CG iteration, 5 per refinement residual
                extra.append(launched - 6 * st.cg_iters - 5 * (st.refine_residuals + st.mid_residual_df))
            outs.append((s.get_m(), s.get_p()))
    assert rel_l2(outs[0][0], outs[1][0]) < 1e-6 and rel_l2(outs[0][1], outs[1][1]) < 1e-6
    assert len(set(extra)) == 1, extra


def test_graph_and_host_loop_agree_3d(hc):
    n, L = (32, 16, 16), (1.0, 0.5, 0.5)
    g, r, S, m0 = _problem(n, L)
    out = []
    for use_graph in (True, False):
        with solver(hc, n, L, "fp32_refined", c=5.0, D=0.03, use_graph=use_graph) as s:
            s.set_r(r)
            s.set_source(S)
            s.set_m(m0)
            st = s.step(5)
            out.append((s.get_m(), s.get_p(), st.total_cg_iters, st.total_sweeps))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2:] == out[1][2:]


def test_batch_mixes_2d_and_3d_contexts(hc):
    """One graph launch per step advances a 2D and a 3D context; each ends
    bit-identical to stepping it alone."""
    probs = [((32, 32), (1.0, 1.0)), ((16, 16, 16), (1.0, 1.0, 1.0))]
    def make(n, L):
        s = solver(hc, n, L, "fp32_refined", c=5.0, D=0.03)
        g = O.Grid(n, L)
        s.set_r(np.full(g.shape, 0.1))
        s.set_source(W.minus_mean(W.gaussian(n, (0.5,) * len(n), 0.1, L)))
        s.set_m(W.uniform_m(g.shape, len(n), 0.0, 0.5, 3))
        return s
    alone = []
    for n, L in probs:
        with make(n, L) as s:
            s.step(3)
            alone.append(s.get_m())
    ss = [make(n, L) for n, L in probs]
    with hc.Batch(ss) as b:
        b.step(3)
    for s, ref in zip(ss, alone):
        assert np.array_equal(s.get_m(), ref)
        s.close()


def test_3d_unsupported_and_invalid_requests(hc):
    import ctypes as C
    from paper_2606_06720_gb300 import _binding as Bd
    with solver(hc, (8, 8, 8), precision="fp32_refined") as s:
        with pytest.raises(hc.HuCaiError) as e:
            s.adjoint(1, np.zeros((3, 8, 8, 8)), 1)
        assert e.value.code == hc.HC_ENOTSUP
        t = Bd.hc_tuning()
        assert Bd.hc_get_tuning(s.ctx, C.byref(t)) == hc.HC_OK
        assert Bd.hc_set_tuning(s.ctx, C.byref(t)) == hc.HC_ENOTSUP
        buf = np.zeros(2 * 512)
        assert Bd.hc_set_m(s.ctx, buf.ctypes.data_as(C.POINTER(C.c_double)), 2 * 512) == hc.HC_EINVAL
    for bad in [(8, 8, 4), (8, 2048, 8), (12, 8, 8)]:
        with pytest.raises(hc.HuCaiError) as e:
            solver(hc, bad)
        assert e.value.code == hc.HC_EINVAL


@pytest.mark.parametrize("precision", ["fp32_refined", "fp32_refined_df"])
def test_source_sink_256_cubed_first_step(hc, precision):
    """The 256^3 source/sink workload in the launch configuration the
    benchmark times (graph mode, cg_rtol 1e-8): after one step the pressure
    satisfies ||S - A(m0) p|| <= 1e-8 ||S|| with A the oracle's FP64
    operator, and the new m equals the oracle's split step (activation,
    relaxation, diffusion of eq. 2.3) applied to the FP32 m0 with that p."""
    w = W.source_sink_3d(256)
    g = O.Grid(w.n, w.L)
    with solver(hc, w.n, w.L, precision, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=1e-8) as s:
        s.set_r(w.r)
        s.set_source(w.S)
        s.set_m(w.m0)
        st = s.step(1)
        assert st.status == hc.HC_OK
        p = s.get_p()
        m1 = s.get_m()
    m0 = w.m0.astype(np.float32).astype(np.float64)
    r32 = w.r.astype(np.float32).astype(np.float64)
    Sp = O.project(g, w.S)
    res = Sp - O.apply_A(g, m0, r32, p)
    assert np.linalg.norm(res) <= 1e-8 * np.linalg.norm(Sp)
    gp = O.gradient(g, p)
    ref = O.diffusion(g, O.relaxation(O.activation(m0, gp, w.c, w.dt), w.gamma, w.dt), w.D, w.dt)
    assert rel_l2(m1, ref) < 2e-6
