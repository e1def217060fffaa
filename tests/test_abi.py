"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point declared in include/hc.h, and validates arguments on the
host before touching the GPU.  No kernel runs here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    return C.CDLL(path)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hc_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hc_create", "hc_set_r", "hc_set_source", "hc_set_m", "hc_set_p", "hc_step",
                     "hc_get_p", "hc_get_m", "hc_destroy", "hc_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_workspace_size_without_gpu(lib):
    from paper_2606_06720_gb300 import _binding as Bd
    assert Bd.strerror(0) == "ok"
    assert "invalid" in Bd.strerror(-1)
    g = Bd.hc_grid(2, (C.c_int * 3)(64, 32, 1), (C.c_double * 3)(1.0, 1.0, 1.0))
    for prec in (Bd.HC_FP64_PLAIN, Bd.HC_FP32_REFINED):
        p = Bd.hc_params(10.0, 0.05, 0.75, 1e-3, 1e-10, 100, prec, 0.0, 1e-4, 10, 0, None)
        nb = C.c_size_t()
        assert Bd.hc_workspace_size(C.byref(g), C.byref(p), C.byref(nb)) == 0
        assert nb.value > 64 * 32 * 8 * 6


@pytest.mark.parametrize("n", [(14, 8), (2, 8), (8, 8192), (64, 0), (3, 3), (49, 50), (5000, 50)])
def test_invalid_grids_are_rejected_on_the_host(lib, n):
    from paper_2606_06720_gb300 import _binding as Bd
    g = Bd.hc_grid(2, (C.c_int * 3)(n[0], n[1], 1), (C.c_double * 3)(1.0, 1.0, 1.0))
    p = Bd.hc_params(10.0, 0.05, 0.75, 1e-3, 1e-10, 100, 0, 0.0, 1e-4, 10, 0, None)
    nb = C.c_size_t()
    assert Bd.hc_workspace_size(C.byref(g), C.byref(p), C.byref(nb)) == Bd.HC_EINVAL
    ctx = C.c_void_p()
    assert Bd.hc_create(C.byref(ctx), C.byref(g), C.byref(p), None, 0) == Bd.HC_EINVAL
    assert not ctx.value


def test_invalid_params_are_rejected_on_the_host(lib):
    from paper_2606_06720_gb300 import _binding as Bd
    g = Bd.hc_grid(2, (C.c_int * 3)(16, 16, 1), (C.c_double * 3)(1.0, 1.0, 1.0))
    ctx = C.c_void_p()
    bad = [Bd.hc_params(10.0, 0.05, 0.75, 1e-3, 1e-10, 100, 7, 0.0, 1e-4, 10, 0, None),
           Bd.hc_params(float("nan"), 0.05, 0.75, 1e-3, 1e-10, 100, 0, 0.0, 1e-4, 10, 0, None),
           Bd.hc_params(10.0, 0.05, 0.75, -1.0, 1e-10, 100, 0, 0.0, 1e-4, 10, 0, None)]
    for p in bad:
        assert Bd.hc_create(C.byref(ctx), C.byref(g), C.byref(p), None, 0) == Bd.HC_EINVAL
    # misaligned borrowed workspace
    p = Bd.hc_params(10.0, 0.05, 0.75, 1e-3, 1e-10, 100, 0, 0.0, 1e-4, 10, 0, None)
    assert Bd.hc_create(C.byref(ctx), C.byref(g), C.byref(p), C.c_void_p(4097), 1 << 30) == Bd.HC_EINVAL
    # null context pointers
    assert Bd.hc_step(None, 1, None) == Bd.HC_EINVAL
    assert Bd.hc_set_r(None, None, 0) == Bd.HC_EINVAL


def test_precond_and_refinement_options_on_the_host(lib):
    """The preconditioner option takes the two values of reading R3 only, and
    the FP64-refined mode's workspace holds, beyond the double-float mode's,
    the double-float copy of S that its mid-step residual reads and the
    buffers of the lagged certification: m of the step awaiting it and of the
    step in flight (4 FP32 fields), its pressure and its two FP64 gradient
    fields (3 FP64 spectra), and its own partial sums (8 doubles per CTA of the
    largest reducing grid, at least 1216) and solve state."""
    from paper_2606_06720_gb300 import _binding as Bd
    n = (64, 32)
    g = Bd.hc_grid(2, (C.c_int * 3)(n[0], n[1], 1), (C.c_double * 3)(1.0, 1.0, 1.0))

    def params(**kw):
        p = Bd.hc_params(10.0, 0.05, 0.75, 1e-3, 1e-10, 100, Bd.HC_FP32_REFINED, 0.0, 1e-4, 10, 0,
                         None)
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    nb = C.c_size_t()
    for pc in (Bd.HC_PRECOND_SCALAR, Bd.HC_PRECOND_KBAR):
        assert Bd.hc_workspace_size(C.byref(g), C.byref(params(precond=pc)), C.byref(nb)) == 0
    ctx = C.c_void_p()
    for pc in (2, -1):
        assert Bd.hc_workspace_size(C.byref(g), C.byref(params(precond=pc)), C.byref(nb)) == Bd.HC_EINVAL
        assert Bd.hc_create(C.byref(ctx), C.byref(g), C.byref(params(precond=pc)), None, 0) == Bd.HC_EINVAL
    sizes = {}
    for prec in (Bd.HC_FP32_REFINED, Bd.HC_FP32_REFINED_DF):
        assert Bd.hc_workspace_size(C.byref(g), C.byref(params(precision=prec)), C.byref(nb)) == 0
        sizes[prec] = nb.value
    extra = sizes[Bd.HC_FP32_REFINED] - sizes[Bd.HC_FP32_REFINED_DF]
    spec16 = n[0] // 2 * n[1] * 16                       # one packed spectrum of 16-byte values
    fixed = spec16 + 4 * n[0] * n[1] * 4 + 3 * spec16 + 8 * 8 * max(n[0] // 2, n[1], 1216)
    assert fixed < extra <= fixed + 4096 + 8 * 256       # + the solve state, alignment


# --- the bounds-checked build (libhc_gb300_check.so, HC_CHECK=1) -------------------------------

@pytest.fixture(scope="module")
def lib_check(lib):
    import __graft_entry__
    return C.CDLL(__graft_entry__._builder().LIB_CHECK)


def test_checked_library_exports_every_declared_symbol(lib_check):
    missing = [n for n in declared_functions() if not hasattr(lib_check, n)]
    assert not missing, missing


def _workspace_bytes(l, n, precision):
    from paper_2606_06720_gb300 import _binding as Bd
    l.hc_workspace_size.argtypes = [C.POINTER(Bd.hc_grid), C.POINTER(Bd.hc_params),
                                    C.POINTER(C.c_size_t)]
    g = Bd.hc_grid(len(n), (C.c_int * 3)(*(tuple(n) + (1,) * (3 - len(n)))),
                   (C.c_double * 3)(1.0, 1.0, 1.0))
    p = Bd.hc_params(10.0, 0.05, 0.75, 1e-3, 1e-10, 100, precision, 0.0, 1e-4, 10, 0, None)
    nb = C.c_size_t()
    assert l.hc_workspace_size(C.byref(g), C.byref(p), C.byref(nb)) == 0
    return nb.value


@pytest.mark.parametrize("n", [(64, 32), (16, 16, 16)])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_checked_workspace_carries_a_guard_zone_per_buffer(lib, lib_check, n, precision):
    """Every buffer of the checked build is followed by HC_REDZONE_BYTES of
    guard zone: the workspace grows by at least that much per buffer (the
    context carves more than 30 buffers)."""
    extra = _workspace_bytes(lib_check, n, precision) - _workspace_bytes(lib, n, precision)
    assert extra >= 30 * 65536
    assert extra % 256 == 0


def test_check_entry_points_without_a_context(lib, lib_check):
    for l in (lib, lib_check):
        l.hc_check_redzones.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_size_t)]
        l.hc_check_poke.argtypes = [C.c_void_p, C.c_int]
        nz, zone, owner = C.c_int(7), C.c_int(7), C.c_size_t(7)
        assert l.hc_check_redzones(None, C.byref(nz), C.byref(zone), C.byref(owner)) == -1
        assert (nz.value, zone.value, owner.value) == (0, -1, 0)
        assert l.hc_check_redzones(None, None, None, None) == -1
    assert lib.hc_check_poke(None, 0) == -7        # HC_ENOTSUP: the product build has no zones
    assert lib_check.hc_check_poke(None, 0) == -1  # HC_EINVAL: no context


def test_hc_check_changes_only_the_host_orchestration():
    """The checked library links the product's kernel objects and recompiles
    only hc_api.cu. That holds while no other translation unit, and no header
    they include, tests HC_CHECK."""
    csrc = os.path.join(ROOT, "paper_2606_06720_gb300", "csrc")
    users = [f for f in sorted(os.listdir(csrc)) if "HC_CHECK" in open(os.path.join(csrc, f)).read()]
    assert users == ["hc_api.cu"]
    header = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "hc.h")).read(), flags=re.S)
    assert "HC_CHECK" not in header


def test_binding_marshals_host_buffers_without_a_gpu(lib):
    """_host_f64: FP64 C-contiguous arrays pass through, others are copied for
    inputs and refused for outputs; sizes are checked; torch CPU tensors must
    be contiguous FP64."""
    import numpy as np
    import torch
    from paper_2606_06720_gb300 import _binding as Bd
    a = np.arange(12, dtype=np.float64).reshape(3, 4)
    p, keep = Bd._host_f64(a, 12)
    assert keep is a
    p, keep = Bd._host_f64(a.T, 12)                     # non-contiguous input: copied
    assert keep is not a and keep.flags["C_CONTIGUOUS"] and np.array_equal(keep, a.T)
    p, keep = Bd._host_f64(a.astype(np.float32), 12)    # other dtype: converted
    assert keep.dtype == np.float64
    with pytest.raises(ValueError):
        Bd._host_f64(a.T, 12, writable=True)            # an output must be written in place
    with pytest.raises(ValueError):
        Bd._host_f64(a, 13)
    t = torch.zeros(12, dtype=torch.float64)
    p, keep = Bd._host_f64(t, 12)
    assert keep is t
    for bad in (torch.zeros(12, dtype=torch.float32), torch.zeros(4, 6, dtype=torch.float64).t()):
        with pytest.raises(ValueError):
            Bd._host_f64(bad, 12)


def test_error_codes_and_messages(lib):
    from paper_2606_06720_gb300 import _binding as Bd
    codes = [Bd.HC_OK, Bd.HC_EINVAL, Bd.HC_ENOMEM, Bd.HC_ECUDA, Bd.HC_ENOCONV, Bd.HC_ENONFINITE,
             Bd.HC_ETIMEOUT, Bd.HC_ENOTSUP, Bd.HC_EBOUNDS]
    assert codes == [0, -1, -2, -3, -4, -5, -6, -7, -8]
    msgs = [Bd.strerror(c) for c in codes]
    assert len(set(msgs)) == len(msgs) and "unknown" not in " ".join(msgs)
    assert "guard zone" in Bd.strerror(Bd.HC_EBOUNDS)
    assert Bd.strerror(-99) == "unknown error"
    err = Bd.HuCaiError(Bd.HC_EBOUNDS, "hc_check_redzones")
    assert "hc_check_redzones" in str(err) and err.code == -8
    with pytest.raises(Bd.HuCaiError):
        Bd._check(Bd.HC_EINVAL, "x")
    Bd._check(Bd.HC_ENOCONV, "x", ok=(Bd.HC_OK, Bd.HC_ENOCONV))


def test_grid_validation_matches_the_documented_rule(lib):
    """hc_workspace_size accepts a grid exactly when include/hc.h says the
    library supports it: 2D axes in [4, 4096] with no prime factor above 5
    (FP64 plain unless both are powers of two in [8, 4096]); 3D axes powers of
    two in [8, 1024] with at most 2^28 points; lengths positive and finite."""
    hyp = pytest.importorskip("hypothesis")
    from hypothesis import given, settings, strategies as st
    from paper_2606_06720_gb300 import _binding as Bd

    def pow2_in(v, lo, hi):
        return lo <= v <= hi and (v & (v - 1)) == 0

    def smooth_in(v, lo, hi):  # no prime factor above 5
        if not lo <= v <= hi:
            return False
        for p in (2, 3, 5):
            while v % p == 0:
                v //= p
        return v == 1

    def supported(dim, n, L, precision):
        if not all(x > 0 and x != float("inf") for x in L[:dim]):
            return False
        if dim == 2:
            if not (smooth_in(n[0], 4, 4096) and smooth_in(n[1], 4, 4096) and n[2] == 1):
                return False
            return precision == 0 or (pow2_in(n[0], 8, 4096) and pow2_in(n[1], 8, 4096))
        return all(pow2_in(v, 8, 1024) for v in n) and n[0] * n[1] * n[2] <= 1 << 28

    axis = st.sampled_from([0, 1, 4, 6, 7, 8, 12, 14, 16, 50, 64, 1000, 1024, 2048, 4096, 8192])
    length = st.sampled_from([1.0, 0.25, 0.0, -1.0, float("inf")])

    @settings(max_examples=400, deadline=None, derandomize=True)
    @given(st.sampled_from([2, 3]), axis, axis, axis, length, length, length, st.sampled_from([0, 1]))
    def check(dim, a, b, c, la, lb, lc, precision):
        n = (a, b, c if dim == 3 else 1)
        L = (la, lb, lc if dim == 3 else 1.0)
        g = Bd.hc_grid(dim, (C.c_int * 3)(*n), (C.c_double * 3)(*L))
        p = Bd.hc_params(10.0, 0.05, 0.75, 1e-3, 1e-10, 100, precision, 0.0, 1e-4, 10, 0, None)
        nb = C.c_size_t()
        rc = Bd.hc_workspace_size(C.byref(g), C.byref(p), C.byref(nb))
        assert (rc == 0) == supported(dim, n, L, precision), (dim, n, L, precision, rc)
        if rc != 0:
            assert rc in (Bd.HC_EINVAL, Bd.HC_ENOTSUP)

    check()


def test_param_validation_matches_the_documented_rule(lib):
    """hc_params is accepted exactly when precision is one of the three modes,
    precond one of the two options, and c, D, gamma, dt are finite with dt >= 0."""
    pytest.importorskip("hypothesis")
    import math
    from hypothesis import given, settings, strategies as st
    from paper_2606_06720_gb300 import _binding as Bd
    val = st.sampled_from([0.0, 1.0, -2.5, 1e-3, float("nan"), float("inf"), -float("inf")])

    @settings(max_examples=300, deadline=None, derandomize=True)
    @given(val, val, val, val, st.integers(-1, 3), st.integers(-1, 2))
    def check(c, D, gamma, dt, precision, precond):
        g = Bd.hc_grid(2, (C.c_int * 3)(64, 32, 1), (C.c_double * 3)(1.0, 1.0, 1.0))
        p = Bd.hc_params(c, D, gamma, dt, 1e-10, 100, precision, 0.0, 1e-4, 10, 0, None,
                         0, 0, 0, precond)
        nb = C.c_size_t()
        rc = Bd.hc_workspace_size(C.byref(g), C.byref(p), C.byref(nb))
        ok = (precision in (0, 1, 2) and precond in (0, 1)
              and all(math.isfinite(x) for x in (c, D, gamma, dt)) and dt >= 0)
        assert (rc == 0) == ok, (c, D, gamma, dt, precision, precond, rc)

    check()


def test_state_calls_reject_a_null_context(lib):
    """hc_set_state / hc_get_state check their arguments before any copy: a
    NULL context (or NULL buffers) is HC_EINVAL on the host."""
    from paper_2606_06720_gb300 import _binding as Bd
    import numpy as np
    m, p = np.zeros(2 * 64), np.zeros(64)
    dp = C.POINTER(C.c_double)
    pm, pp = m.ctypes.data_as(dp), p.ctypes.data_as(dp)
    assert Bd.hc_set_state(None, pm, m.size, pp, p.size) == Bd.HC_EINVAL
    assert Bd.hc_get_state(None, pm, m.size, pp, p.size) == Bd.HC_EINVAL
    assert Bd.hc_set_state(None, dp(), m.size, dp(), p.size) == Bd.HC_EINVAL
