"""hc_spectrum_noalloc: the forward transform for callers that cannot allocate
device memory (a plugin inside a framework that reserves the whole GPU for its
own pool, or a loop that cannot afford cudaMalloc's implicit synchronisation).
Its scratch is a fixed static device array; its output must equal that of the
existing entry point hc_spectrum, on two calls in a row.

Kept in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

import oracle as O  # noqa: F401  (gpu_common sets the oracle's threads)
from gpu_common import hc, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu


def test_noalloc_spectrum_matches_hc_spectrum_on_two_calls(hc):
    import torch
    from paper_2606_06720_gb300 import _binding as Bd
    rng = np.random.default_rng(31)
    stream = torch.cuda.current_stream()
    # each call is smaller than one before it: anything it read from an
    # earlier call's scratch contents instead of its own would show up.  The
    # extreme aspect ratios take the shared-memory opt-in of the row pass
    # (4096 x 16) and a column tile clamped to one column (16 x 4096).
    for nx, ny in [(256, 256), (4096, 16), (16, 4096), (64, 32), (8, 8)]:
        f = rng.standard_normal((ny, nx))
        with hc.Solver((nx, ny), (1.0, 1.0), c=1.0, D=0.1, gamma=1.0, dt=1e-3,
                       precision="fp64") as s:
            ref = s.spectrum(f)  # existing entry point
        fd = torch.from_numpy(f).cuda()
        out = torch.full((ny * (nx // 2) * 2,), float("nan"), dtype=torch.float64, device="cuda")
        rc = Bd.hc_spectrum_noalloc(C.c_void_p(fd.data_ptr()), C.c_void_p(out.data_ptr()), nx, ny,
                                    C.c_void_p(stream.cuda_stream))
        assert rc == hc.HC_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.complex128).reshape(ny, nx // 2)
        assert rel_l2(got, ref) < 1e-12


def test_noalloc_spectrum_rejects_sizes_beyond_its_scratch(hc):
    import torch
    from paper_2606_06720_gb300 import _binding as Bd
    fd = torch.zeros(4, dtype=torch.float64, device="cuda")
    for nx, ny in [(512, 256), (4096, 4096), (12, 8), (8, 8192)]:
        assert Bd.hc_spectrum_noalloc(C.c_void_p(fd.data_ptr()), C.c_void_p(fd.data_ptr()), nx, ny,
                                      None) == hc.HC_EINVAL
    assert Bd.hc_spectrum_noalloc(None, None, 64, 64, None) == hc.HC_EINVAL
