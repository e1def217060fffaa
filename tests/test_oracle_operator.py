"""Pins for the oracle's pressure operator (eq. 1.1a, eq. p_discrete), the
null-space projection, the preconditioner and preconditioned CG (Section 2.4).

Pins: the tensor's eigenstructure (Section 1.1), the constant-coefficient
closed form (m = 0), a manufactured solution derived symbolically from
eq. (1.1a) with sympy, and a dense 8x8 assembly solved by numpy's
least-squares routine.
"""
import numpy as np
import pytest
import sympy as sp

import oracle as O

RNG = np.random.default_rng(99)


def test_tensor_eigenstructure():
    """(m (x) m + r I) has eigenvalue r + |m|^2 along m and r along m-perp."""
    npts = 50
    m = RNG.standard_normal((2, npts))
    r = RNG.uniform(0.05, 0.3, npts)
    q = O.apply_K(m, r, m)
    assert np.allclose(q, (r + (m ** 2).sum(0)) * m, rtol=1e-14, atol=1e-14)
    mperp = np.stack([-m[1], m[0]])
    assert np.allclose(O.apply_K(m, r, mperp), r * mperp, rtol=1e-14, atol=1e-14)
    m3 = RNG.standard_normal((3, npts))
    v = np.cross(m3.T, RNG.standard_normal((npts, 3))).T  # orthogonal to m3
    assert np.allclose(O.apply_K(m3, r, v), r * v, atol=1e-13)


@pytest.mark.parametrize("n,L", [((16, 8), (1.0, 2.0)), ((8, 32), (0.5, 1.0))])
def test_constant_coefficient_operator_closed_form(n, L):
    """m = 0, r = const: A p = r (-Laplacian) p with symbol r |xi~|^2."""
    g = O.Grid(n, L)
    r0 = 0.37
    m = np.zeros((2,) + g.shape)
    r = np.full(g.shape, r0)
    # single mode: A cos(2 pi (k x / Lx + l y / Ly)) = r (2 pi)^2 ((k/Lx)^2 + (l/Ly)^2) cos(...)
    X, Y = np.meshgrid(np.arange(n[0]) * L[0] / n[0], np.arange(n[1]) * L[1] / n[1])
    k, l = 3, 2
    p = np.cos(2 * np.pi * (k * X / L[0] + l * Y / L[1]))
    lam = r0 * (2 * np.pi) ** 2 * ((k / L[0]) ** 2 + (l / L[1]) ** 2)
    assert np.allclose(O.apply_A(g, m, r, p), lam * p, atol=1e-11 * lam)
    # random field versus the same symbol applied with numpy's FFT
    p = RNG.standard_normal(g.shape)
    lx = np.arange(n[0]); ly = np.arange(n[1])
    xix = np.where(lx < n[0] // 2, 2 * np.pi * lx / L[0], np.where(lx == n[0] // 2, 0.0, 2 * np.pi * (lx - n[0]) / L[0]))
    xiy = np.where(ly < n[1] // 2, 2 * np.pi * ly / L[1], np.where(ly == n[1] // 2, 0.0, 2 * np.pi * (ly - n[1]) / L[1]))
    sym = r0 * (xix[None, :] ** 2 + xiy[:, None] ** 2)
    ref = np.fft.ifft2(sym * np.fft.fft2(p)).real
    assert np.allclose(O.apply_A(g, m, r, p), ref, atol=1e-10)


def manufactured(n, L):
    """p, m, r band-limited trig polynomials; S = -div((m m^T + r I) grad p)
    computed symbolically from eq. (1.1a)."""
    x, y = sp.symbols("x y", real=True)
    Lx, Ly = [sp.nsimplify(v) for v in L]
    tx, ty = 2 * sp.pi * x / Lx, 2 * sp.pi * y / Ly
    p = sp.sin(tx) * sp.cos(2 * ty) + sp.Rational(1, 2) * sp.cos(tx + ty)
    m1 = sp.Rational(3, 10) + sp.Rational(1, 5) * sp.cos(ty)
    m2 = sp.Rational(2, 5) * sp.sin(tx)
    r = sp.Rational(1, 10) + sp.Rational(1, 20) * sp.cos(tx)
    px, py = sp.diff(p, x), sp.diff(p, y)
    mg = m1 * px + m2 * py
    q1 = m1 * mg + r * px
    q2 = m2 * mg + r * py
    S = -(sp.diff(q1, x) + sp.diff(q2, y))
    f = sp.lambdify((x, y), (p, m1, m2, r, S), "numpy")
    X, Y = np.meshgrid(np.arange(n[0]) * L[0] / n[0], np.arange(n[1]) * L[1] / n[1])
    vals = [np.broadcast_to(np.asarray(v, dtype=float), X.shape).copy() for v in f(X, Y)]
    P, M1, M2, R, S = vals
    return P, np.stack([M1, M2]), R, S


@pytest.mark.parametrize("n,L", [((16, 16), (1.0, 1.0)), ((16, 32), (1.0, 2.0)),
                                 ((32, 16), (0.5, 1.0))])
def test_operator_manufactured_solution(n, L):
    g = O.Grid(n, L)
    P, M, R, S = manufactured(n, L)
    Ap = O.apply_A(g, M, R, P)
    assert np.abs(Ap - S).max() < 1e-11 * np.abs(S).max()


@pytest.mark.parametrize("n,L", [((16, 16), (1.0, 1.0)), ((32, 16), (0.5, 1.0))])
def test_pcg_recovers_manufactured_pressure(n, L):
    g = O.Grid(n, L)
    P, M, R, S = manufactured(n, L)
    b = O.project(g, S)
    x, st = O.pcg(g, M, R, b, rtol=1e-13, maxit=500)
    assert st.rc == O.OK
    Pp = O.project(g, P)
    assert np.allclose(Pp, P, atol=1e-14)  # P has no null-mode content
    assert np.abs(x - Pp).max() < 1e-10 * np.abs(P).max()


def assemble(g, m, r):
    n = g.npts
    A = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = O.apply_A(g, m, r, e.reshape(g.shape)).ravel()
    return A


def corner_modes(g):
    ny, nx = g.shape
    i = np.arange(nx); j = np.arange(ny)
    out = []
    for ex in (0, 1):
        for ey in (0, 1):
            out.append((((-1.0) ** (ex * i))[None, :] * ((-1.0) ** (ey * j))[:, None]).ravel())
    return np.array(out)


def test_dense_8x8_symmetric_psd_nullspace_and_solve():
    g = O.Grid((8, 8), (1.0, 1.5))
    m = RNG.uniform(0, 1, (2,) + g.shape)
    r = RNG.uniform(0.05, 0.2, g.shape)
    A = assemble(g, m, r)
    assert np.abs(A - A.T).max() < 1e-11 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() > -1e-10 * ev.max()
    assert (np.abs(ev) < 1e-9 * ev.max()).sum() == 4  # R2: exactly the corner modes
    C = corner_modes(g)
    assert np.abs(A @ C.T).max() < 1e-10 * np.abs(A).max()
    # projection removes exactly the corner-mode components
    f = RNG.standard_normal(g.shape)
    Q, _ = np.linalg.qr(C.T)
    fp_ref = f.ravel() - Q @ (Q.T @ f.ravel())
    assert np.allclose(O.project(g, f).ravel(), fp_ref, atol=1e-13)
    # CG versus the minimum-norm least-squares solution
    S = O.project(g, RNG.standard_normal(g.shape))
    x_ls = np.linalg.lstsq(A, S.ravel(), rcond=1e-12)[0]
    x_cg, st = O.pcg(g, m, r, S, rtol=1e-13, maxit=500)
    assert st.rc == O.OK
    assert np.abs(x_cg.ravel() - x_ls).max() < 1e-9 * np.abs(x_ls).max()


@pytest.mark.parametrize("n", [(9, 4), (5, 7)])
def test_projection_on_odd_grids_is_the_projector_onto_the_range(n):
    """An odd axis has no Nyquist index, so its alternating mode is not a
    null mode. The operator's null space, from the SVD of its dense
    assembly, is then the constants plus the Nyquist modes of the even axes.
    project() must be the orthogonal projector onto its complement."""
    g = O.Grid(n, (1.0, 0.7))
    m = RNG.uniform(0, 1, (2,) + g.shape)
    r = RNG.uniform(0.05, 0.2, g.shape)
    A = assemble(g, m, r)
    U, sv, _ = np.linalg.svd(A)
    null = U[:, sv < 1e-9 * sv.max()]
    assert null.shape[1] == (2 if (n[0] % 2 == 0 or n[1] % 2 == 0) else 1)
    f = RNG.standard_normal(g.shape).ravel()
    want = f - null @ (null.T @ f)
    assert np.allclose(O.project(g, f.reshape(g.shape)).ravel(), want, atol=1e-12)


def test_pcg_reports_the_residual_it_reached():
    """The reported relative residual is ||S - A x||_2 / ||S||_2 of the
    returned x, recomputed here with numpy's norm (reading R4)."""
    g = O.Grid((16, 8), (1.0, 0.5))
    m = RNG.uniform(0, 1, (2,) + g.shape)
    r = RNG.uniform(0.05, 0.2, g.shape)
    S = O.project(g, RNG.standard_normal(g.shape))
    for rtol in (1e-3, 1e-9):
        x, st = O.pcg(g, m, r, S, rtol=rtol)
        res = np.linalg.norm(S - O.apply_A(g, m, r, x)) / np.linalg.norm(S)
        assert st.true_rel_residual == pytest.approx(res, rel=1e-6, abs=1e-15)
        assert st.rel_residual == pytest.approx(res, rel=1e-3)   # recurrence vs recomputed
        assert res <= rtol * 1.01


def test_pcg_constant_coefficient_converges_in_one_iteration():
    g = O.Grid((16, 32), (1.0, 2.0))
    r0 = 0.2
    m = np.zeros((2,) + g.shape)
    r = np.full(g.shape, r0)
    S = O.project(g, RNG.standard_normal(g.shape))
    x, st = O.pcg(g, m, r, S, kappa=r0, rtol=1e-12, maxit=10)
    assert st.rc == O.OK and st.cg_iters == 1
    # closed form: p^ = S^ / (r |xi~|^2) off the null modes
    n = g.n
    lx = np.arange(n[0]); ly = np.arange(n[1])
    xix = np.where(lx < n[0] // 2, 2 * np.pi * lx / 1.0, np.where(lx == n[0] // 2, 0.0, 2 * np.pi * (lx - n[0]) / 1.0))
    xiy = np.where(ly < n[1] // 2, 2 * np.pi * ly / 2.0, np.where(ly == n[1] // 2, 0.0, 2 * np.pi * (ly - n[1]) / 2.0))
    sym = r0 * (xix[None, :] ** 2 + xiy[:, None] ** 2)
    Sh = np.fft.fft2(S)
    ph = np.where(sym > 0, Sh / np.where(sym > 0, sym, 1), 0)
    assert np.allclose(x, np.fft.ifft2(ph).real, atol=1e-12)


def test_pcg_constant_anisotropic_coefficient_converges_in_one_iteration():
    """With constant m and r the anisotropic option of reading R3,
    -div(Kbar grad) with Kbar = mean(m m^T) + mean(r) I = K, is the operator
    itself: one iteration, and the closed form p^ = S^ / (xi~^T K xi~) off the
    null modes."""
    g = O.Grid((16, 32), (1.0, 2.0))
    mc, r0 = np.array([0.6, -0.3]), 0.15
    m = np.broadcast_to(mc[:, None, None], (2,) + g.shape).copy()
    r = np.full(g.shape, r0)
    S = O.project(g, RNG.standard_normal(g.shape))
    x, st = O.pcg(g, m, r, S, rtol=1e-12, maxit=10, precond=1)
    assert st.rc == O.OK and st.cg_iters == 1
    # the default (isotropic kappa) preconditioner is not exact here
    assert O.pcg(g, m, r, S, rtol=1e-12, maxit=10)[1].cg_iters > 1
    n = g.n
    lx = np.arange(n[0]); ly = np.arange(n[1])
    xix = np.where(lx < n[0] // 2, 2 * np.pi * lx / 1.0, np.where(lx == n[0] // 2, 0.0, 2 * np.pi * (lx - n[0]) / 1.0))
    xiy = np.where(ly < n[1] // 2, 2 * np.pi * ly / 2.0, np.where(ly == n[1] // 2, 0.0, 2 * np.pi * (ly - n[1]) / 2.0))
    X, Y = xix[None, :], xiy[:, None]
    sym = (mc[0] * X + mc[1] * Y) ** 2 + r0 * (X ** 2 + Y ** 2)
    Sh = np.fft.fft2(S)
    ph = np.where(sym > 0, Sh / np.where(sym > 0, sym, 1), 0)
    assert np.allclose(x, np.fft.ifft2(ph).real, atol=1e-12)
    # kappa is reported as trace(Kbar) / dim
    assert st.kappa == pytest.approx(r0 + (mc ** 2).sum() / 2, rel=1e-14)


def test_preconditioner_on_single_mode_3d():
    """One Fourier mode cos(xi . x) is an eigenfunction of -div(Kbar grad) with
    eigenvalue xi^T Kbar xi (xi written out by hand, off the Nyquist indices)."""
    g = O.Grid((8, 16, 8), (1.0, 2.0, 0.5))
    K = np.array([[0.5, 0.1, -0.2], [0.1, 0.4, 0.05], [-0.2, 0.05, 0.3]])
    kvec = np.array([1, 3, 2])  # mode indices along x, y, z
    xi = 2 * np.pi * kvec / np.array(g.L)
    xs = [np.arange(n) * (Lx / n) for n, Lx in zip(g.n, g.L)]
    Z, Yg, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    f = np.cos(xi[0] * X + xi[1] * Yg + xi[2] * Z)
    z = O.precond(g, K, f)
    assert np.allclose(z, f / (xi @ K @ xi), atol=1e-12)


@pytest.mark.parametrize("precond", [0, 1])
def test_pcg_iterations_within_condition_bound(precond):
    """Generalised eigenvalues of (A, -div(Kbar grad)) lie between the extreme
    pointwise eigenvalues of Kbar^-1/2 K(x) Kbar^-1/2, so the CG error bound
    gives it <= ceil(sqrt(cond)/2 * ln(2/rtol)); both preconditioners of
    reading R3."""
    g = O.Grid((32, 32))
    m = RNG.uniform(0, 1, (2,) + g.shape)
    r = RNG.uniform(0.05, 0.15, g.shape)
    S = O.project(g, RNG.standard_normal(g.shape))
    rtol = 1e-10
    kb = O.kbar_default(g, m, r) if precond else O.kbar_array(2, O.kappa_default(g, m, r))
    Kbar = np.array([[kb[0], kb[3]], [kb[3], kb[1]]])
    w, V = np.linalg.eigh(Kbar)
    Kih = V @ np.diag(w ** -0.5) @ V.T
    K = np.einsum("a...,b...->...ab", m, m) + r[..., None, None] * np.eye(2)
    lam = np.linalg.eigvalsh(Kih @ K @ Kih)
    cond = lam.max() / lam.min()
    # bound on ||e||_A; relative residual picks up at most sqrt(cond(A)) more
    condA = cond * (w.max() / w.min()) * (2 * np.pi * 16) ** 2 / (2 * np.pi) ** 2
    bound = int(np.ceil(0.5 * np.sqrt(cond) * np.log(2 * np.sqrt(condA) / rtol)))
    x, st = O.pcg(g, m, r, S, rtol=rtol, maxit=10000, precond=precond)
    assert st.rc == O.OK
    assert st.cg_iters <= bound
    assert st.true_rel_residual < 10 * rtol


def test_pcg_warm_start_at_solution_takes_no_iteration():
    g = O.Grid((16, 16))
    m = RNG.uniform(0, 1, (2,) + g.shape)
    r = np.full(g.shape, 0.1)
    S = O.project(g, RNG.standard_normal(g.shape))
    x, st = O.pcg(g, m, r, S, rtol=1e-12)
    x2, st2 = O.pcg(g, m, r, S, x0=x, rtol=1e-10)
    assert st2.cg_iters == 0
    assert np.array_equal(x2, O.project(g, x))


def test_pcg_stopping_rule_is_relative_to_the_source():
    """Reading R4: CG stops at ||S - A p||_2 <= rtol ||S||_2. The rule is relative, so
    scaling S by a power of two scales every iterate exactly. The iteration count and the
    result are then unchanged up to that factor. An absolute rule would stop the scaled
    problems at other counts."""
    g = O.Grid((16, 16))
    m = RNG.uniform(0, 1, (2,) + g.shape)
    r = np.full(g.shape, 0.1)
    S = O.project(g, RNG.standard_normal(g.shape))
    x, st = O.pcg(g, m, r, S, rtol=1e-10)
    assert st.rc == 0
    for k in (-30, 30):
        s = 2.0 ** k
        xs, sts = O.pcg(g, m, r, s * S, rtol=1e-10)
        assert sts.rc == 0 and sts.cg_iters == st.cg_iters
        assert np.array_equal(xs, s * x)
        assert sts.rel_residual == st.rel_residual


def test_pcg_zero_source_gives_zero_pressure():
    g = O.Grid((8, 8))
    m = RNG.uniform(0, 1, (2,) + g.shape)
    r = np.full(g.shape, 0.1)
    x, st = O.pcg(g, m, r, np.zeros(g.shape), x0=RNG.standard_normal(g.shape))
    assert st.cg_iters == 0 and np.all(x == 0)


def test_preconditioner_inverts_constant_coefficient_operator():
    g = O.Grid((16, 8), (1.0, 2.0))
    kappa = 0.7
    m = np.zeros((2,) + g.shape)
    r = np.full(g.shape, kappa)
    p = O.project(g, RNG.standard_normal(g.shape))
    z = O.precond(g, kappa, O.apply_A(g, m, r, p))
    assert np.allclose(z, p, atol=1e-12)
    # null modes map to zero
    C = corner_modes(g)
    for c in C:
        assert np.abs(O.precond(g, kappa, c.reshape(g.shape))).max() < 1e-14


def manufactured_3d(n, L):
    """3D analogue of `manufactured`: band-limited p, m (3 components), r and
    S = -div((m m^T + r I) grad p) from eq. (1.1a), symbolically."""
    x, y, z = sp.symbols("x y z", real=True)
    Lx, Ly, Lz = [sp.nsimplify(v) for v in L]
    tx, ty, tz = 2 * sp.pi * x / Lx, 2 * sp.pi * y / Ly, 2 * sp.pi * z / Lz
    p = sp.sin(tx) * sp.cos(ty + tz) + sp.Rational(1, 3) * sp.cos(2 * tz - tx)
    m = [sp.Rational(3, 10) + sp.Rational(1, 5) * sp.cos(tz),
         sp.Rational(2, 5) * sp.sin(tx),
         sp.Rational(1, 4) * sp.cos(ty)]
    r = sp.Rational(1, 10) + sp.Rational(1, 20) * sp.sin(ty)
    grad = [sp.diff(p, v) for v in (x, y, z)]
    mg = sum(mi * gi for mi, gi in zip(m, grad))
    q = [mi * mg + r * gi for mi, gi in zip(m, grad)]
    S = -(sp.diff(q[0], x) + sp.diff(q[1], y) + sp.diff(q[2], z))
    f = sp.lambdify((x, y, z), (p, *m, r, S), "numpy")
    Z, Y, X = np.meshgrid(np.arange(n[2]) * L[2] / n[2], np.arange(n[1]) * L[1] / n[1],
                          np.arange(n[0]) * L[0] / n[0], indexing="ij")
    vals = [np.broadcast_to(np.asarray(v, dtype=float), X.shape).copy() for v in f(X, Y, Z)]
    P, M1, M2, M3, R, S = vals
    return P, np.stack([M1, M2, M3]), R, S


@pytest.mark.parametrize("n,L", [((16, 16, 16), (1.0, 1.0, 1.0)), ((16, 8, 32), (1.0, 0.5, 2.0))])
def test_operator_manufactured_solution_3d(n, L):
    g = O.Grid(n, L)
    P, M, R, S = manufactured_3d(n, L)
    assert np.abs(O.apply_A(g, M, R, P) - S).max() < 1e-11 * np.abs(S).max()
    x, st = O.pcg(g, M, R, O.project(g, S), rtol=1e-13, maxit=500)
    assert st.rc == O.OK
    assert np.abs(x - P).max() < 1e-10 * np.abs(P).max()


def test_dense_3d_symmetric_psd_with_eight_null_modes():
    """Reading R2 in 3D: with the Nyquist first-derivative multiplier zeroed,
    N(A) is spanned by the 8 modes whose wavenumbers are all 0 or N/2."""
    g = O.Grid((4, 4, 4), (1.0, 0.5, 2.0))
    m = RNG.uniform(-1, 1, (3,) + g.shape)
    r = RNG.uniform(0.1, 0.3, g.shape)
    A = assemble(g, m, r)
    assert np.allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    w = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert w.min() > -1e-12 * w.max()
    assert int((w > 1e-10 * w.max()).sum()) == 64 - 8
    k = np.arange(4)
    for ex in (0, 1):
        for ey in (0, 1):
            for ez in (0, 1):
                v = (((-1.0) ** (ex * k))[None, None, :] * ((-1.0) ** (ey * k))[None, :, None]
                     * ((-1.0) ** (ez * k))[:, None, None]).ravel()
                assert np.abs(A @ v).max() < 1e-12 * np.abs(A).max()
                assert np.abs(O.project(g, v.reshape(g.shape))).max() < 1e-14


def test_constant_coefficient_operator_closed_form_3d():
    g = O.Grid((8, 16, 8), (1.0, 2.0, 0.5))
    r0 = 0.2
    Z, Y, X = np.meshgrid(np.arange(8) * 0.5 / 8, np.arange(16) * 2.0 / 16, np.arange(8) / 8,
                          indexing="ij")
    p = np.cos(2 * np.pi * (1 * X + 3 * Y / 2.0 + 2 * Z / 0.5))
    lam = r0 * (2 * np.pi) ** 2 * (1 + (3 / 2.0) ** 2 + (2 / 0.5) ** 2)
    m = np.zeros((3,) + g.shape)
    Ap = O.apply_A(g, m, np.full(g.shape, r0), p)
    assert np.allclose(Ap, lam * p, atol=1e-11 * lam)
