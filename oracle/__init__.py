"""Plain FP64 CPU oracle of the Fourier spectral FFT+CG splitting scheme for the
periodic Hu-Cai system (arXiv 2606.06720, Section 2 and Algorithm 1).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The GPU product path
(``paper_2606_06720_gb300``) never imports it, and this package never imports
the product.  The arithmetic lives in ``hc_oracle.c`` (plain C, FP64); this
module only marshals numpy arrays through ctypes.

Array conventions: a scalar field on a 2D grid has numpy shape ``(ny, nx)``
(3D: ``(nz, ny, nx)``), x fastest; a vector field has a leading component axis,
``(dim, ny, nx)``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hc_oracle.c")
_HDR = os.path.join(_HERE, "hc_oracle.h")
_LIB = os.path.join(_HERE, "libhc_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENOCONV, ENONFINITE = 0, -1, -2, -4, -5


def build(force: bool = False) -> str:
    """Compile hc_oracle.c into libhc_oracle.so (gcc, FP64, no FMA contraction
    so x86 and Arm hosts round identically)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3)]


class _Params(C.Structure):
    _fields_ = [("c", C.c_double), ("D", C.c_double), ("gamma", C.c_double), ("dt", C.c_double),
                ("cg_rtol", C.c_double), ("cg_maxit", C.c_int), ("kappa", C.c_double),
                ("precond", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("cg_iters", C.c_int), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double), ("kappa", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # HC_ORACLE_LIB names another build of hc_oracle.c: the test that
            # plants mistakes in copies of the source loads those builds.
            lib = C.CDLL(os.environ.get("HC_ORACLE_LIB") or build())
            dp = C.POINTER(C.c_double)
            gp = C.POINTER(_Grid)
            lib.or_set_threads.argtypes = [C.c_int]
            lib.or_get_threads.restype = C.c_int
            lib.or_dft1.argtypes = [dp, dp, C.c_int, C.c_int]
            lib.or_fft1.argtypes = [dp, C.c_int, C.c_int]
            lib.or_fftn.argtypes = [gp, dp, C.c_int]
            lib.or_xi.argtypes = [C.c_int, C.c_int, C.c_double]
            lib.or_xi.restype = C.c_double
            lib.or_xi_deriv.argtypes = [C.c_int, C.c_int, C.c_double]
            lib.or_xi_deriv.restype = C.c_double
            lib.or_gradient.argtypes = [gp, dp, dp]
            lib.or_apply_K.argtypes = [C.c_int, C.c_size_t, dp, dp, dp, dp]
            lib.or_apply_K.restype = None
            lib.or_apply_A.argtypes = [gp, dp, dp, dp, dp]
            lib.or_precond.argtypes = [gp, dp, dp, dp]
            lib.or_kbar_default.argtypes = [gp, dp, dp, dp]
            lib.or_kbar_default.restype = None
            lib.or_project.argtypes = [gp, dp]
            lib.or_project.restype = None
            lib.or_kappa_default.argtypes = [gp, dp, dp]
            lib.or_kappa_default.restype = C.c_double
            lib.or_pcg.argtypes = [gp, dp, dp, dp, dp, dp, C.c_double, C.c_int,
                                   C.POINTER(_Stats)]
            lib.or_activation.argtypes = [C.c_int, C.c_size_t, dp, dp, C.c_double, C.c_double]
            lib.or_activation.restype = None
            lib.or_relaxation.argtypes = [C.c_int, C.c_size_t, dp, C.c_double, C.c_double]
            lib.or_relaxation.restype = None
            lib.or_diffusion.argtypes = [gp, dp, C.c_double, C.c_double]
            lib.or_step.argtypes = [gp, C.POINTER(_Params), dp, dp, dp, dp, C.POINTER(_Stats)]
            lib.or_energy.argtypes = [gp, C.POINTER(_Params), dp, dp, dp]
            lib.or_energy.restype = C.c_double
            lib.or_adjoint.argtypes = [gp, C.POINTER(_Params), dp, dp, dp, dp, C.c_int, dp, dp, dp,
                                       dp, dp, dp]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check(rc: int, what: str):
    if rc not in (OK,):
        raise RuntimeError(f"oracle {what} failed with code {rc}")


@dataclass(frozen=True)
class Grid:
    """Uniform periodic grid: ``n = (nx, ny[, nz])`` nodes, lengths ``L``."""
    n: tuple
    L: tuple = None

    def __post_init__(self):
        if self.L is None:
            object.__setattr__(self, "L", tuple(1.0 for _ in self.n))

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def shape(self) -> tuple:
        return tuple(reversed(self.n))

    @property
    def npts(self) -> int:
        return int(np.prod(self.n))

    def c(self) -> _Grid:
        g = _Grid()
        g.dim = self.dim
        for a in range(3):
            g.n[a] = self.n[a] if a < self.dim else 1
            g.L[a] = self.L[a] if a < self.dim else 1.0
        return g


@dataclass
class Params:
    c: float
    D: float
    gamma: float
    dt: float
    cg_rtol: float = 1e-10
    cg_maxit: int = 1000
    kappa: float = 0.0
    precond: int = 0   # 0: kappa (-Laplacian), reading R3; 1: the anisotropic Kbar option

    def c_struct(self) -> _Params:
        return _Params(self.c, self.D, self.gamma, self.dt, self.cg_rtol, int(self.cg_maxit),
                       self.kappa, int(self.precond))


@dataclass
class Stats:
    cg_iters: int
    rel_residual: float
    true_rel_residual: float
    kappa: float
    rc: int = 0


def _stats(s: _Stats, rc: int = 0) -> Stats:
    return Stats(s.cg_iters, s.rel_residual, s.true_rel_residual, s.kappa, rc)


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def get_threads() -> int:
    return _load().or_get_threads()


def dft1(a, sign: int = -1) -> np.ndarray:
    x = _c128(a)
    out = np.empty_like(x)
    _check(_load().or_dft1(_dp(x.view(np.float64)), _dp(out.view(np.float64)), x.size, sign), "dft1")
    return out


def fft1(a, sign: int = -1) -> np.ndarray:
    x = _c128(a).copy()
    _check(_load().or_fft1(_dp(x.view(np.float64)), x.size, sign), "fft1")
    return x


def fftn(grid: Grid, a, sign: int = -1) -> np.ndarray:
    """sign=-1: unnormalised forward transform; sign=+1: inverse with 1/npts."""
    x = _c128(a).reshape(grid.shape).copy()
    g = grid.c()
    _check(_load().or_fftn(C.byref(g), _dp(x.view(np.float64)), sign), "fftn")
    return x


def xi(l: int, N: int, L: float = 1.0) -> float:
    return _load().or_xi(l, N, L)


def xi_deriv(l: int, N: int, L: float = 1.0) -> float:
    return _load().or_xi_deriv(l, N, L)


def gradient(grid: Grid, f) -> np.ndarray:
    f = _f64(f).reshape(grid.shape)
    out = np.empty((grid.dim,) + grid.shape)
    g = grid.c()
    _check(_load().or_gradient(C.byref(g), _dp(f), _dp(out)), "gradient")
    return out


def apply_K(m, r, v) -> np.ndarray:
    m, r, v = _f64(m), _f64(r), _f64(v)
    dim = m.shape[0]
    q = np.empty_like(v)
    _load().or_apply_K(dim, r.size, _dp(m), _dp(r), _dp(v), _dp(q))
    return q


def apply_A(grid: Grid, m, r, p) -> np.ndarray:
    m, r, p = _f64(m), _f64(r), _f64(p)
    out = np.empty(grid.shape)
    g = grid.c()
    _check(_load().or_apply_A(C.byref(g), _dp(m), _dp(r), _dp(p), _dp(out)), "apply_A")
    return out


def kbar_array(dim: int, kbar) -> np.ndarray:
    """The preconditioner matrix in the oracle's layout (xx, yy, zz, xy, xz, yz)
    from a scalar kappa (kappa I), a dim x dim symmetric matrix, or the
    6-vector itself."""
    a = np.asarray(kbar, dtype=np.float64)
    if a.ndim == 0:
        return np.array([float(a) if e < dim else 0.0 for e in range(6)])
    if a.shape == (6,):
        return a.copy()
    M = np.zeros((3, 3))
    M[:dim, :dim] = a
    return np.array([M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]])


def precond(grid: Grid, kbar, res) -> np.ndarray:
    """z = F^-1[F(res) / (xi~^T Kbar xi~)] (reading R3); kbar as in kbar_array."""
    res = _f64(res)
    out = np.empty(grid.shape)
    g = grid.c()
    kb = kbar_array(grid.dim, kbar)
    _check(_load().or_precond(C.byref(g), _dp(kb), _dp(res), _dp(out)), "precond")
    return out


def kbar_default(grid: Grid, m, r) -> np.ndarray:
    """The default preconditioner matrix mean(m m^T) + mean(r) I (reading R3),
    as the 6-vector xx, yy, zz, xy, xz, yz."""
    m, r = _f64(m), _f64(r)
    out = np.zeros(6)
    g = grid.c()
    _load().or_kbar_default(C.byref(g), _dp(m), _dp(r), _dp(out))
    return out


def project(grid: Grid, f) -> np.ndarray:
    x = _f64(f).reshape(grid.shape).copy()
    g = grid.c()
    _load().or_project(C.byref(g), _dp(x))
    return x


def kappa_default(grid: Grid, m, r) -> float:
    m, r = _f64(m), _f64(r)
    g = grid.c()
    return _load().or_kappa_default(C.byref(g), _dp(m), _dp(r))


def pcg(grid: Grid, m, r, b, x0=None, kappa=None, rtol: float = 1e-10, maxit: int = 1000,
        precond: int = 0):
    """Returns (x, Stats); raises nothing on non-convergence (Stats.rc says).
    kappa: None for reading R3's preconditioner (precond 0: kappa_default I;
    precond 1: kbar_default), else a scalar kappa (kappa I), a dim x dim
    matrix or the 6-vector of kbar_array."""
    m, r, b = _f64(m), _f64(r), _f64(b)
    x = np.zeros(grid.shape) if x0 is None else _f64(x0).reshape(grid.shape).copy()
    if kappa is None:
        kb = kbar_default(grid, m, r) if precond == 1 else kbar_array(grid.dim, kappa_default(grid, m, r))
    else:
        kb = kbar_array(grid.dim, kappa)
    st = _Stats()
    g = grid.c()
    rc = _load().or_pcg(C.byref(g), _dp(m), _dp(r), _dp(b), _dp(x), _dp(kb), rtol, int(maxit),
                        C.byref(st))
    if rc not in (OK, ENOCONV):
        _check(rc, "pcg")
    return x, _stats(st, rc)


def activation(m, grad_p, c: float, dt: float) -> np.ndarray:
    m2 = _f64(m).copy()
    g = _f64(grad_p)
    dim = m2.shape[0]
    _load().or_activation(dim, m2[0].size, _dp(m2), _dp(g), c, dt)
    return m2


def relaxation(m, gamma: float, dt: float) -> np.ndarray:
    m2 = _f64(m).copy()
    dim = m2.shape[0]
    _load().or_relaxation(dim, m2[0].size, _dp(m2), gamma, dt)
    return m2


def diffusion(grid: Grid, m, D: float, dt: float) -> np.ndarray:
    m2 = _f64(m).reshape((grid.dim,) + grid.shape).copy()
    g = grid.c()
    _check(_load().or_diffusion(C.byref(g), _dp(m2), D, dt), "diffusion")
    return m2


def step(grid: Grid, prm: Params, r, S, m, p):
    """One loop body of Algorithm 1.  Returns (m_new, p_new, Stats).  A step
    that left NaN/Inf in m (the activation exponential overflowed, Remark 2.1)
    returns that state with Stats.rc = ENONFINITE, as the library reports it;
    invalid arguments raise."""
    r, S = _f64(r), _f64(S)
    m2 = _f64(m).reshape((grid.dim,) + grid.shape).copy()
    p2 = _f64(p).reshape(grid.shape).copy()
    st = _Stats()
    g = grid.c()
    cp = prm.c_struct()
    rc = _load().or_step(C.byref(g), C.byref(cp), _dp(r), _dp(S), _dp(m2), _dp(p2), C.byref(st))
    if rc not in (OK, ENOCONV, ENONFINITE):
        _check(rc, "step")
    return m2, p2, _stats(st, rc)


def energy(grid: Grid, prm: Params, r, m, p) -> float:
    r, m, p = _f64(r), _f64(m), _f64(p)
    g = grid.c()
    cp = prm.c_struct()
    return _load().or_energy(C.byref(g), C.byref(cp), _dp(r), _dp(m), _dp(p))


def adjoint(grid: Grid, prm: Params, r, S, m0, p0, nsteps: int, lamT):
    """Discrete adjoint of `nsteps` steps: returns dict with dc2, dD2 (floats)
    and dr, dS (fields), dm0 (vector field), for dL/dm(T) = lamT."""
    r, S = _f64(r), _f64(S)
    m0 = _f64(m0).reshape((grid.dim,) + grid.shape)
    p0 = _f64(p0).reshape(grid.shape)
    lamT = _f64(lamT).reshape((grid.dim,) + grid.shape)
    dc2, dD2 = C.c_double(), C.c_double()
    dr, dS = np.empty(grid.shape), np.empty(grid.shape)
    dm0 = np.empty((grid.dim,) + grid.shape)
    g = grid.c()
    cp = prm.c_struct()
    _check(_load().or_adjoint(C.byref(g), C.byref(cp), _dp(r), _dp(S), _dp(m0), _dp(p0),
                              int(nsteps), _dp(lamT), C.byref(dc2), C.byref(dD2), _dp(dr),
                              _dp(dS), _dp(dm0)), "adjoint")
    return {"dc2": dc2.value, "dD2": dD2.value, "dr": dr, "dS": dS, "dm0": dm0}


def delta_m(m_new, m_old, dt: float) -> float:
    """Relative change of the conductivity per unit time (Section 2.5):
    ||m^k - m^{k-1}||_2 / (dt ||m^{k-1}||_2), discrete L2 norms (the cell
    volume cancels in the ratio).  Reading R20: 0 when m^{k-1} = 0, a steady
    state (every substep maps m = 0 to 0), where the ratio is 0/0."""
    m_new, m_old = _f64(m_new), _f64(m_old)
    old2 = (m_old ** 2).sum()
    if old2 == 0:
        return 0.0
    return float(np.sqrt(((m_new - m_old) ** 2).sum() / old2) / dt)


@dataclass
class RunResult:
    m: np.ndarray
    p: np.ndarray
    steps: int
    reason: int             # 0 max steps, 1 delta m <= eps, 2 energy not decreasing, 3 failed step
    energies: list          # energies[k] = E_h(m^k) with its own pressure p[m^k]
    delta_ms: list          # delta_ms[k] = Delta m of the step m^k -> m^{k+1}
    energy_step: int = -1   # reason 2: the step whose result did not lower the energy


def run(grid: Grid, prm: Params, r, S, m0, p0=None, max_steps: int = 1000, eps: float = 1e-4,
        stop_on_energy: bool = True) -> RunResult:
    """Algorithm 1's while loop with the two stopping rules of Section 2.5:
    loop bodies continue while Delta m > eps (eps <= 0: never stop on it) and
    the discrete energy decreases, at most max_steps of them.

    The energy is read as a function of m alone, E_h(m) with the pressure
    that solves eq. (1.1a) for that m.  The loop body from m^k solves exactly
    that pressure, so E_h(m^k) becomes known in step k (0-based), and the
    energy rule E_h(m^k) >= E_h(m^{k-1}) is applied after step k; it then
    names step k-1 (the one that produced m^k) in energy_step.  The Delta m
    rule is applied first.  Returns the state after the last step run."""
    m = _f64(m0).reshape((grid.dim,) + grid.shape).copy()
    p = np.zeros(grid.shape) if p0 is None else _f64(p0).reshape(grid.shape).copy()
    energies, dms = [], []
    reason, energy_step, steps = 0, -1, 0
    for k in range(max_steps):
        m_new, p, st = step(grid, prm, r, S, m, p)  # p = p[m^k]
        steps = k + 1
        if st.rc not in (OK, ENOCONV) or not np.isfinite(m_new).all():
            m, reason = m_new, 3
            break
        energies.append(energy(grid, prm, r, m, p))
        dms.append(delta_m(m_new, m, prm.dt))
        m = m_new
        if eps > 0 and dms[-1] <= eps:
            reason = 1
            break
        if stop_on_energy and len(energies) >= 2 and not energies[-1] < energies[-2]:
            reason, energy_step = 2, k - 1
            break
    return RunResult(m, p, steps, reason, energies, dms, energy_step)
