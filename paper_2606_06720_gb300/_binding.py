"""ctypes binding of ``include/hc.h``: argument marshalling only.

The module-level functions carry the C names (``hc_create``, ``hc_step`` ...)
and take/return plain ctypes values.  ``Solver`` wraps one context: it
allocates the device workspace as a torch tensor, passes torch's current CUDA
stream, and converts numpy / torch CPU arrays to the FP64 host pointers the
ABI expects.  Nothing here computes any part of the scheme.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# HC_GB300_CHECK=1 in the environment loads the bounds-checked build instead
# (same kernels; guard zones after every workspace buffer, see hc_check_redzones).
CHECKED = os.environ.get("HC_GB300_CHECK", "0") == "1"
_LIBNAME = os.path.join(HERE, "libhc_gb300_check.so" if CHECKED else "libhc_gb300.so")

HC_OK, HC_EINVAL, HC_ENOMEM, HC_ECUDA = 0, -1, -2, -3
HC_ENOCONV, HC_ENONFINITE, HC_ETIMEOUT, HC_ENOTSUP, HC_EBOUNDS = -4, -5, -6, -7, -8
HC_FP64_PLAIN, HC_FP32_REFINED, HC_FP32_REFINED_DF = 0, 1, 2
HC_STOP_NONE, HC_STOP_DELTA_M, HC_STOP_ENERGY, HC_STOP_STATUS = 0, 1, 2, 3
HC_PRECOND_SCALAR, HC_PRECOND_KBAR = 0, 1


class HuCaiError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        detail = ""
        if code == HC_ECUDA:
            detail = " [" + lib.hc_last_cuda_error().decode() + "]"
        super().__init__(f"{what}: {strerror(code)} ({code}){detail}")


class hc_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3)]


# preconditioner of reading R3: "scalar" kappa (-Laplacian) (the default) or
# "kbar", the whole mean of the coefficient tensor
_PRECOND = {"scalar": HC_PRECOND_SCALAR, "kbar": HC_PRECOND_KBAR}


class hc_params(C.Structure):
    _fields_ = [("c", C.c_double), ("D", C.c_double), ("gamma", C.c_double), ("dt", C.c_double),
                ("cg_rtol", C.c_double), ("cg_maxit", C.c_int), ("precision", C.c_int),
                ("kappa", C.c_double), ("inner_rtol", C.c_double), ("max_sweeps", C.c_int),
                ("use_graph", C.c_int), ("stream", C.c_void_p), ("diagnostics", C.c_int),
                ("fp64_first_residual", C.c_int), ("fp64_mid_residual", C.c_int),
                ("precond", C.c_int), ("sync_cert", C.c_int)]


class hc_tuning(C.Structure):
    _fields_ = [("col_tile", C.c_int * 2), ("row_rows", C.c_int * 2), ("col_pipe", C.c_int * 2),
                ("row_pipe", C.c_int * 2)]


class hc_step_stats(C.Structure):
    _fields_ = [("cg_iters", C.c_int), ("refine_sweeps", C.c_int), ("rel_residual", C.c_double),
                ("kappa", C.c_double), ("status", C.c_int), ("total_cg_iters", C.c_longlong),
                ("total_sweeps", C.c_longlong), ("energy", C.c_double), ("delta_m", C.c_double),
                ("energy_valid", C.c_int), ("stop_reason", C.c_int), ("energy_step", C.c_longlong),
                ("first_sweep_fp32", C.c_int), ("total_first_fp32", C.c_longlong),
                ("mid_residual_df", C.c_int), ("total_mid_df", C.c_longlong),
                ("refine_residuals", C.c_int), ("total_refine_residuals", C.c_longlong)]


def library_path() -> str:
    return _LIBNAME


def _load() -> C.CDLL:
    if not os.path.exists(_LIBNAME):
        raise ImportError(
            f"{_LIBNAME} is missing: build it with `python -m paper_2606_06720_gb300.build` "
            "(or __graft_entry__.build()); there is no CPU fallback")
    lib = C.CDLL(_LIBNAME)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    sig = {
        "hc_workspace_size": ([C.POINTER(hc_grid), C.POINTER(hc_params), C.POINTER(C.c_size_t)], C.c_int),
        "hc_create": ([C.POINTER(P), C.POINTER(hc_grid), C.POINTER(hc_params), P, C.c_size_t], C.c_int),
        "hc_set_params": ([P, C.POINTER(hc_params)], C.c_int),
        "hc_set_r": ([P, dp, C.c_size_t], C.c_int),
        "hc_set_source": ([P, dp, C.c_size_t], C.c_int),
        "hc_set_m": ([P, dp, C.c_size_t], C.c_int),
        "hc_set_p": ([P, dp, C.c_size_t], C.c_int),
        "hc_step": ([P, C.c_int, C.POINTER(hc_step_stats)], C.c_int),
        "hc_run": ([P, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(hc_step_stats)],
                   C.c_int),
        "hc_get_p": ([P, dp, C.c_size_t], C.c_int),
        "hc_get_m": ([P, dp, C.c_size_t], C.c_int),
        "hc_set_state": ([P, dp, C.c_size_t, dp, C.c_size_t], C.c_int),
        "hc_get_state": ([P, dp, C.c_size_t, dp, C.c_size_t], C.c_int),
        "hc_gradient": ([P, dp, C.c_size_t], C.c_int),
        "hc_apply_operator": ([P, dp, dp, C.c_size_t], C.c_int),
        "hc_split_step": ([P], C.c_int),
        "hc_spectrum": ([P, dp, dp, C.c_size_t], C.c_int),
        "hc_launch_count": ([P, C.POINTER(C.c_longlong)], C.c_int),
        "hc_fp64_fma_peak": ([C.c_int, P, dp], C.c_int),
        "hc_destroy": ([P], None),
        "hc_strerror": ([C.c_int], C.c_char_p),
        "hc_last_cuda_error": ([], C.c_char_p),
        "hc_time_kernel": ([P, C.c_int, C.c_int, dp], C.c_int),
        "hc_get_tuning": ([P, C.POINTER(hc_tuning)], C.c_int),
        "hc_set_tuning": ([P, C.POINTER(hc_tuning)], C.c_int),
        "hc_spectrum_noalloc": ([P, P, C.c_int, C.c_int, P], C.c_int),
        "hc_adjoint_workspace_size": ([P, C.c_int, C.c_int, C.POINTER(C.c_size_t)], C.c_int),
        "hc_adjoint": ([P, C.c_int, C.c_int, dp, dp, dp, dp, dp, dp, P, C.c_size_t], C.c_int),
        "hc_batch_create": ([C.POINTER(P), C.POINTER(P), C.c_int, P], C.c_int),
        "hc_batch_step": ([P, C.c_int, C.POINTER(hc_step_stats)], C.c_int),
        "hc_batch_destroy": ([P], None),
        "hc_batch_classes": ([P, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
        "hc_check_redzones": ([P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)],
                              C.c_int),
        "hc_check_poke": ([P, C.c_int], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()

# C-named entry points (thin aliases) ----------------------------------------
hc_workspace_size = lib.hc_workspace_size
hc_create = lib.hc_create
hc_set_params = lib.hc_set_params
hc_set_r = lib.hc_set_r
hc_set_source = lib.hc_set_source
hc_set_m = lib.hc_set_m
hc_set_p = lib.hc_set_p
hc_step = lib.hc_step
hc_run = lib.hc_run
hc_get_p = lib.hc_get_p
hc_get_m = lib.hc_get_m
hc_set_state = lib.hc_set_state
hc_get_state = lib.hc_get_state
hc_gradient = lib.hc_gradient
hc_apply_operator = lib.hc_apply_operator
hc_split_step = lib.hc_split_step
hc_spectrum = lib.hc_spectrum
hc_launch_count = lib.hc_launch_count
hc_fp64_fma_peak = lib.hc_fp64_fma_peak
hc_destroy = lib.hc_destroy
hc_time_kernel = lib.hc_time_kernel
hc_get_tuning = lib.hc_get_tuning
hc_set_tuning = lib.hc_set_tuning
hc_spectrum_noalloc = lib.hc_spectrum_noalloc
hc_adjoint_workspace_size = lib.hc_adjoint_workspace_size
hc_adjoint = lib.hc_adjoint
hc_batch_create = lib.hc_batch_create
hc_batch_step = lib.hc_batch_step
hc_batch_destroy = lib.hc_batch_destroy
hc_batch_classes = lib.hc_batch_classes
hc_check_redzones = lib.hc_check_redzones
hc_check_poke = lib.hc_check_poke

# kernel ids of hc_time_kernel (include/hc.h)
KERNELS = ["cg_grad", "cg_apply", "cg_div", "cg_update", "res_grad", "res_apply", "res_div",
           "split_grad", "split_row", "split_heat", "split_c2r", "cg_ypass", "res_ypass",
           "first_grad", "first_apply", "first_div", "mid_grad", "mid_apply", "mid_div", "mid_ypass"]


def strerror(code: int) -> str:
    return lib.hc_strerror(int(code)).decode()


def _check(rc: int, what: str, ok=(HC_OK,)):
    if rc not in ok:
        raise HuCaiError(rc, what)
    return rc


@dataclass
class StepStats:
    cg_iters: int
    refine_sweeps: int
    rel_residual: float
    kappa: float
    status: int
    rc: int
    total_cg_iters: int = 0
    total_sweeps: int = 0
    energy: float = 0.0          # E_h of the step's starting m (diagnostics on, energy_valid)
    delta_m: float = 0.0         # Delta m of the step (diagnostics on)
    energy_valid: int = 0
    stop_reason: int = HC_STOP_NONE
    energy_step: int = -1
    steps: int = 0               # Solver.run: steps executed
    first_sweep_fp32: int = 0    # refined: the last step's first sweep started from an FP32 residual
    total_first_fp32: int = 0
    mid_residual_df: int = 0     # fp32_refined: the last step evaluated the double-float mid-step residual
    total_mid_df: int = 0
    refine_residuals: int = 0    # refined: residuals in the mode's refinement arithmetic (last step)
    total_refine_residuals: int = 0


def _stats(st, rc: int, steps: int = 0) -> StepStats:
    return StepStats(st.cg_iters, st.refine_sweeps, st.rel_residual, st.kappa, st.status, rc,
                     st.total_cg_iters, st.total_sweeps, st.energy, st.delta_m, st.energy_valid,
                     st.stop_reason, st.energy_step, steps, st.first_sweep_fp32,
                     st.total_first_fp32, st.mid_residual_df, st.total_mid_df,
                     st.refine_residuals, st.total_refine_residuals)


def _host_f64(a, count: int, writable: bool = False):
    """(pointer, keepalive) of a contiguous FP64 host buffer: numpy array or
    torch CPU tensor (pinned or not)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != count:
                raise ValueError("expected a contiguous float64 CPU tensor of %d elements" % count)
            return C.cast(C.c_void_p(a.data_ptr()), C.POINTER(C.c_double)), a
    except ImportError:
        pass
    arr = np.asarray(a)
    if arr.dtype != np.float64 or not arr.flags["C_CONTIGUOUS"]:
        if writable:
            raise ValueError("output buffer must be a contiguous float64 array")
        arr = np.ascontiguousarray(arr, dtype=np.float64)
    if arr.size != count:
        raise ValueError("expected %d elements, got %d" % (count, arr.size))
    return arr.ctypes.data_as(C.POINTER(C.c_double)), arr


class Solver:
    """One Hu-Cai problem on one GPU.

    ``n = (nx, ny)`` or ``(nx, ny, nz)`` nodes, ``L`` the domain lengths (same
    length); ``precision`` is ``"fp64"`` (plain), ``"fp32_refined"`` (FP64
    refinement) or ``"fp32_refined_df"`` (refinement in double-float on the FP32
    pipes).  Arrays use numpy shapes ``(ny, nx)`` / ``(nz, ny, nx)`` for scalar
    fields and ``(dim, ...)`` for m and the gradient.
    """

    def __init__(self, n, L=None, *, c: float, D: float, gamma: float, dt: float,
                 precision: str = "fp32_refined", cg_rtol: float = 1e-8, cg_maxit: int = 1000,
                 kappa: float = 0.0, inner_rtol: float = 1e-4, max_sweeps: int = 10,
                 use_graph: bool = True, device: str = "cuda:0", stream=None,
                 diagnostics: bool = False, fp64_first_residual: bool = False,
                 fp64_mid_residual: bool = False, precond: str = "scalar",
                 sync_cert: bool = False):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.dim = len(n)
        if self.dim not in (2, 3):
            raise ValueError("n must have 2 or 3 entries")
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in (L if L is not None else (1.0,) * self.dim))
        if len(self.L) != self.dim:
            raise ValueError("L must have as many entries as n")
        self.npts = int(np.prod(self.n))
        self.shape = tuple(reversed(self.n))
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        n3 = self.n + (1,) * (3 - self.dim)
        L3 = self.L + (1.0,) * (3 - self.dim)
        self.grid = hc_grid(self.dim, (C.c_int * 3)(*n3), (C.c_double * 3)(*L3))
        prec = {"fp64": HC_FP64_PLAIN, "fp64_plain": HC_FP64_PLAIN,
                "fp32_refined": HC_FP32_REFINED, "fp32_refined_df": HC_FP32_REFINED_DF}[precision]
        self.precision = precision
        self.params = hc_params(c, D, gamma, dt, cg_rtol, int(cg_maxit), prec, kappa, inner_rtol,
                                int(max_sweeps), int(bool(use_graph)), self.stream.cuda_stream,
                                int(bool(diagnostics)), int(bool(fp64_first_residual)),
                                int(bool(fp64_mid_residual)), _PRECOND[precond],
                                int(bool(sync_cert)))
        nbytes = C.c_size_t()
        _check(hc_workspace_size(C.byref(self.grid), C.byref(self.params), C.byref(nbytes)),
               "hc_workspace_size")
        # device memory comes from torch's allocator; the context borrows it
        self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(hc_create(C.byref(self.ctx), C.byref(self.grid), C.byref(self.params),
                             C.c_void_p(aligned), nbytes.value), "hc_create")

    # lifecycle -----------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            hc_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # parameters and fields ----------------------------------------------
    def set_params(self, **kw):
        for k, v in kw.items():
            if k in ("use_graph", "diagnostics", "fp64_first_residual", "fp64_mid_residual",
                     "sync_cert"):
                v = int(bool(v))
            if k == "precond":
                v = _PRECOND[v] if isinstance(v, str) else int(v)
            setattr(self.params, k, v)
        _check(hc_set_params(self.ctx, C.byref(self.params)), "hc_set_params")

    def set_r(self, r):
        p, keep = _host_f64(r, self.npts)
        _check(hc_set_r(self.ctx, p, self.npts), "hc_set_r")

    def set_source(self, S):
        p, keep = _host_f64(S, self.npts)
        _check(hc_set_source(self.ctx, p, self.npts), "hc_set_source")

    def set_m(self, m):
        p, keep = _host_f64(m, self.dim * self.npts)
        _check(hc_set_m(self.ctx, p, self.dim * self.npts), "hc_set_m")

    def set_p(self, p_):
        p, keep = _host_f64(p_, self.npts)
        _check(hc_set_p(self.ctx, p, self.npts), "hc_set_p")

    def get_p(self, out=None):
        out = np.empty(self.shape) if out is None else out
        p, keep = _host_f64(out, self.npts, writable=True)
        _check(hc_get_p(self.ctx, p, self.npts), "hc_get_p")
        return out

    def get_m(self, out=None):
        out = np.empty((self.dim,) + self.shape) if out is None else out
        p, keep = _host_f64(out, self.dim * self.npts, writable=True)
        _check(hc_get_m(self.ctx, p, self.dim * self.npts), "hc_get_m")
        return out

    def set_state(self, m, p_):
        """m and p in one call (hc_set_state)."""
        pm, keep_m = _host_f64(m, self.dim * self.npts)
        pp, keep_p = _host_f64(p_, self.npts)
        _check(hc_set_state(self.ctx, pm, self.dim * self.npts, pp, self.npts), "hc_set_state")

    def get_state(self, m_out=None, p_out=None):
        """(m, p) in one call (hc_get_state); returns the two buffers."""
        m_out = np.empty((self.dim,) + self.shape) if m_out is None else m_out
        p_out = np.empty(self.shape) if p_out is None else p_out
        pm, keep_m = _host_f64(m_out, self.dim * self.npts, writable=True)
        pp, keep_p = _host_f64(p_out, self.npts, writable=True)
        _check(hc_get_state(self.ctx, pm, self.dim * self.npts, pp, self.npts), "hc_get_state")
        return m_out, p_out

    # the step -------------------------------------------------------------
    def step(self, nsteps: int = 1, allow=(HC_OK, HC_ENOCONV)) -> StepStats:
        st = hc_step_stats()
        rc = hc_step(self.ctx, int(nsteps), C.byref(st))
        _check(rc, "hc_step", ok=allow)
        return _stats(st, rc)

    def run(self, max_steps: int, eps: float = 1e-4, stop_on_energy: bool = True,
            allow=(HC_OK, HC_ENOCONV)) -> StepStats:
        """Algorithm 1's loop with its stopping rules (hc_run): until
        Delta m <= eps, the energy stops decreasing, or max_steps."""
        st = hc_step_stats()
        done = C.c_int()
        rc = hc_run(self.ctx, int(max_steps), float(eps), int(bool(stop_on_energy)),
                    C.byref(done), C.byref(st))
        _check(rc, "hc_run", ok=allow)
        return _stats(st, rc, done.value)

    # components ----------------------------------------------------------
    def gradient(self):
        out = np.empty((self.dim,) + self.shape)
        p, keep = _host_f64(out, self.dim * self.npts, writable=True)
        _check(hc_gradient(self.ctx, p, self.dim * self.npts), "hc_gradient")
        return out

    def apply_operator(self, f):
        fp, keep = _host_f64(f, self.npts)
        out = np.empty(self.shape)
        op, keep2 = _host_f64(out, self.npts, writable=True)
        _check(hc_apply_operator(self.ctx, fp, op, self.npts), "hc_apply_operator")
        return out

    def split_step(self):
        _check(hc_split_step(self.ctx), "hc_split_step")

    @property
    def generic(self) -> bool:
        """A 2D grid whose sizes are not both powers of two in [8, 4096]: the
        mixed-radix FP64 path, with the unpacked half spectrum."""
        def pow2(v):
            return 8 <= v <= 4096 and (v & (v - 1)) == 0
        return len(self.n) == 2 and not (pow2(self.n[0]) and pow2(self.n[1]))

    def spectrum(self, f):
        """Packed half spectrum, complex array of shape (ny, nx/2) or (nz, ny, nx/2);
        on a generic-size grid the unpacked half spectrum (ny, nx/2 + 1)."""
        fp, keep = _host_f64(f, self.npts)
        cols = self.n[0] // 2 + 1 if self.generic else self.n[0] // 2
        out = np.empty(self.shape[:-1] + (cols,), dtype=np.complex128)
        op = out.view(np.float64).ctypes.data_as(C.POINTER(C.c_double))
        _check(hc_spectrum(self.ctx, fp, op, self.npts), "hc_spectrum")
        return out

    def time_kernel(self, name: str, reps: int = 20) -> float:
        """Mean milliseconds per launch of one step kernel (see hc_time_kernel)."""
        ms = C.c_double()
        _check(hc_time_kernel(self.ctx, KERNELS.index(name), int(reps), C.byref(ms)),
               "hc_time_kernel")
        return ms.value

    def get_tuning(self) -> dict:
        t = hc_tuning()
        _check(hc_get_tuning(self.ctx, C.byref(t)), "hc_get_tuning")
        return {"col_tile": list(t.col_tile), "row_rows": list(t.row_rows),
                "col_pipe": list(t.col_pipe), "row_pipe": list(t.row_pipe)}

    def set_tuning(self, col_tile, row_rows, col_pipe=None, row_pipe=None):
        cur = self.get_tuning() if col_pipe is None or row_pipe is None else None
        col_pipe = cur["col_pipe"] if col_pipe is None else col_pipe
        row_pipe = cur["row_pipe"] if row_pipe is None else row_pipe
        t = hc_tuning((C.c_int * 2)(*col_tile), (C.c_int * 2)(*row_rows),
                      (C.c_int * 2)(*col_pipe), (C.c_int * 2)(*row_pipe))
        _check(hc_set_tuning(self.ctx, C.byref(t)), "hc_set_tuning")

    def adjoint(self, nsteps: int, lamT, every: int = 50, allow=(HC_OK, HC_ENOCONV)) -> dict:
        """Gradients of a loss on m(T) after `nsteps` steps from the current
        state, given lamT = dL/dm(T) (see hc_adjoint).  Leaves the solver at
        the forward state of step `nsteps`."""
        import torch
        nbytes = C.c_size_t()
        _check(hc_adjoint_workspace_size(self.ctx, int(nsteps), int(every), C.byref(nbytes)),
               "hc_adjoint_workspace_size")
        ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        base = (ws.data_ptr() + 255) // 256 * 256
        lp, keep = _host_f64(lamT, 2 * self.npts)
        dc2, dD2 = C.c_double(), C.c_double()
        dr, dS = np.empty(self.shape), np.empty(self.shape)
        dm0 = np.empty((2,) + self.shape)
        dp_ = C.POINTER(C.c_double)
        rc = hc_adjoint(self.ctx, int(nsteps), int(every), lp, C.byref(dc2), C.byref(dD2),
                        dr.ctypes.data_as(dp_), dS.ctypes.data_as(dp_), dm0.ctypes.data_as(dp_),
                        C.c_void_p(base), nbytes.value)
        _check(rc, "hc_adjoint", ok=allow)
        del ws
        return {"dc2": dc2.value, "dD2": dD2.value, "dr": dr, "dS": dS, "dm0": dm0, "rc": rc}

    def check_redzones(self) -> dict:
        """Guard-zone scan of the bounds-checked build (hc_check_redzones):
        {"rc", "zones", "zone", "owner_bytes"}; zones = 0 in the product build."""
        nz, zone, owner = C.c_int(), C.c_int(), C.c_size_t()
        rc = hc_check_redzones(self.ctx, C.byref(nz), C.byref(zone), C.byref(owner))
        return {"rc": rc, "zones": nz.value, "zone": zone.value, "owner_bytes": owner.value}

    def launch_count(self) -> int:
        v = C.c_longlong()
        _check(hc_launch_count(self.ctx, C.byref(v)), "hc_launch_count")
        return v.value


def fp64_fma_peak(reps: int = 5, stream=None) -> float:
    """Measured FP64 FMA throughput of the current device in TFLOP/s
    (hc_fp64_fma_peak): the ALU roof of the FP64 residual kernels."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    v = C.c_double()
    _check(hc_fp64_fma_peak(int(reps), C.c_void_p(s.cuda_stream), C.byref(v)), "hc_fp64_fma_peak")
    return v.value


class Batch:
    """Several Solvers advanced together by one CUDA graph launch per step
    (hc_batch_*): 2D refined solvers of one grid size as a size class of
    batched launches, the others as chains of their own."""

    def __init__(self, solvers, stream=None):
        import torch
        self.solvers = list(solvers)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.solvers[0].device)
        arr = (C.c_void_p * len(self.solvers))(*[s.ctx.value for s in self.solvers])
        self.b = C.c_void_p()
        _check(hc_batch_create(C.byref(self.b), arr, len(self.solvers),
                               C.c_void_p(self.stream.cuda_stream)), "hc_batch_create")

    def classes(self) -> tuple:
        """(size classes, contexts in them) of hc_batch_classes."""
        a, m = C.c_int(), C.c_int()
        _check(hc_batch_classes(self.b, C.byref(a), C.byref(m)), "hc_batch_classes")
        return a.value, m.value

    def step(self, nsteps: int = 1, allow=(HC_OK, HC_ENOCONV)):
        st = (hc_step_stats * len(self.solvers))()
        rc = hc_batch_step(self.b, int(nsteps), st)
        _check(rc, "hc_batch_step", ok=allow)
        return [_stats(x, rc) for x in st]

    def close(self):
        if getattr(self, "b", None) and self.b.value:
            hc_batch_destroy(self.b)
            self.b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _autograd_function():
    import torch

    class HuCaiSteps(torch.autograd.Function):
        """m(T) = nsteps loop bodies of Algorithm 1 from (m0, p = 0) with
        parameters c^2, D^2 and fields r, S, on a Solver; backward calls the
        hand-written adjoint (hc_adjoint).  Inputs and output are CPU float64
        tensors; c2 and D2 are 0-dim tensors."""

        @staticmethod
        def forward(ctx, solver, nsteps, every, c2, D2, r, S, m0):
            ctx.solver, ctx.nsteps, ctx.every = solver, int(nsteps), int(every)
            ctx.inputs = (float(c2), float(D2), r.detach().clone(), S.detach().clone(),
                          m0.detach().clone())
            HuCaiSteps._load(solver, *ctx.inputs)
            solver.step(nsteps)
            return torch.from_numpy(solver.get_m())

        @staticmethod
        def _load(solver, c2, D2, r, S, m0):
            solver.set_params(c=float(np.sqrt(c2)), D=float(np.sqrt(D2)))
            solver.set_r(r.contiguous())
            solver.set_source(S.contiguous())
            solver.set_m(m0.contiguous())
            solver.set_p(np.zeros(solver.shape))

        @staticmethod
        def backward(ctx, grad_m):
            solver = ctx.solver
            HuCaiSteps._load(solver, *ctx.inputs)
            g = solver.adjoint(ctx.nsteps, grad_m.detach().double().contiguous(), ctx.every)
            t = lambda a: torch.as_tensor(a, dtype=torch.float64)
            return (None, None, None, t(g["dc2"]), t(g["dD2"]), t(g["dr"]), t(g["dS"]),
                    t(g["dm0"]))

    return HuCaiSteps


def hucai_steps(solver, nsteps, every, c2, D2, r, S, m0):
    """Differentiable m(T) (torch.autograd); see HuCaiSteps."""
    return _autograd_function().apply(solver, nsteps, every, c2, D2, r, S, m0)
