"""The seeded synthetic inputs (workloads/) follow their stated recipes: the
64² centred-Gaussian problem, the 512²/2048² source/sink problem, the
48-instance parameter sweep, and the 256³ source/sink pair. They draw the same
values on every call, and the smooth r field is the same function at every
resolution."""
import itertools

import numpy as np

import workloads as W


def test_centred_gaussian_recipe():
    w = W.centered_gaussian_2d(64)
    assert w.n == (64, 64) and (w.c, w.D, w.gamma, w.dt, w.cg_rtol) == (10.0, 0.05, 0.75, 1e-3, 1e-10)
    assert np.all(w.r == 0.1)
    assert abs(w.S.mean()) < 1e-15 and np.unravel_index(np.argmax(w.S), w.S.shape) == (32, 32)
    assert w.m0.shape == (2, 64, 64) and w.m0.min() >= 0 and w.m0.max() <= 1
    assert 0.45 < w.m0.mean() < 0.55


def test_source_sink_recipe():
    w = W.source_sink_2d(512)
    assert (w.c, w.D, w.gamma, w.dt) == (25.0, 0.02, 0.5, 5e-4)
    assert w.r.min() >= 0.05 and w.r.max() <= 0.15 + 1e-12
    assert abs(w.S.mean()) < 1e-15
    # the source at (0.3, 0.5), the sink at (0.7, 0.5): x runs along the last axis
    assert np.unravel_index(np.argmax(w.S), w.S.shape) == (256, round(0.3 * 512))
    assert np.unravel_index(np.argmin(w.S), w.S.shape) == (256, round(0.7 * 512))
    assert w.m0.min() >= 0 and w.m0.max() <= 0.5


def test_smooth_r_is_one_field_at_every_resolution():
    coarse = W.source_sink_2d(512).r
    fine = W.source_sink_2d(2048).r
    assert np.allclose(fine[::4, ::4], coarse, atol=1e-12)


def test_sweep_covers_the_parameter_grid():
    ws = [W.sweep_instance(i) for i in range(48)]
    triples = [(w.c, w.D, w.gamma) for w in ws]
    assert triples == list(itertools.product((5.0, 10.0, 25.0, 50.0), (0.01, 0.02, 0.05, 0.1),
                                             (0.5, 0.75, 1.0)))
    sizes = [w.n[0] for w in ws]
    assert all(w.n[0] == w.n[1] for w in ws)
    assert {s: sizes.count(s) for s in set(sizes)} == {128: 16, 256: 16, 512: 16}
    assert all(w.dt == 1e-3 and np.all(w.r == 0.1) and abs(w.S.mean()) < 1e-15 for w in ws)
    # each instance draws m0 from its own seed
    a, b = W.sweep_instance(0).m0, W.sweep_instance(3).m0
    assert a.shape == b.shape and not np.array_equal(a, b)


def test_source_sink_3d_recipe():
    w = W.source_sink_3d(32)
    assert w.n == (32, 32, 32) and (w.c, w.D, w.gamma, w.dt) == (25.0, 0.03, 0.75, 5e-4)
    assert np.all(w.r == 0.1) and abs(w.S.mean()) < 1e-15
    assert w.m0.shape == (3, 32, 32, 32) and w.m0.min() >= 0 and w.m0.max() <= 0.5


def test_seeded_inputs_repeat():
    a, b = W.source_sink_2d(128), W.source_sink_2d(128)
    assert np.array_equal(a.r, b.r) and np.array_equal(a.S, b.S) and np.array_equal(a.m0, b.m0)
    c = W.source_sink_2d(128, seed=1)
    assert not np.array_equal(a.m0, c.m0) and np.array_equal(a.r, c.r)


def test_paper_inputs_at_chosen_nodes():
    """Section 3's analytic inputs evaluated at nodes x = i/N, y = j/N, stored
    at [j, i] (x along the last axis): m^A decays fast along y and slowly
    along x (eq. m_ini_normal), m^B alike in both (eq. m_ini_symm), S_4 has
    its source at the centre and sinks of weight 1/4 at the four (0.2|0.8,
    0.2|0.8) points (eqs. S_4sinks*), S_int its constant sink pi/1000
    (eq. SinternalSink)."""
    import math
    close = lambda a, b: abs(a - b) <= 1e-14 * abs(b)     # libm exp differs in the last bit
    mA = W.paper_m_ini(64, "A")[0]
    assert close(mA[32, 16], math.exp(-50 * 0.25 ** 2))       # x = 0.25, y = 0.5
    assert close(mA[33, 32], math.exp(-1e4 * (1 / 64) ** 2))  # x = 0.5, y = 0.5 + 1/64
    mB = W.paper_m_ini(64, "B")[0]
    assert mB[32, 16] == mB[16, 32] and close(mB[32, 16], math.exp(-50 * 0.25 ** 2))
    S4 = W.paper_S4(10)                                    # nodes at 0.2, 0.5 and 0.8
    assert abs(S4[5, 5] - 1.0) < 1e-70
    for j, i in ((2, 2), (2, 8), (8, 2), (8, 8)):
        assert abs(S4[j, i] + 0.25) < 1e-70
    Si = W.paper_Sint(10)
    assert close(Si[5, 5], 1.0 - math.pi / 1000)
