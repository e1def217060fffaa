"""GB300 (sm_103a) implementation of one time step of the Fourier spectral
FFT+CG splitting scheme for the periodic Hu-Cai network-formation system
(Aceves-Sanchez, Degond, Merino-Aceituno, Wytrzens, arXiv 2606.06720).

Every step of the path runs in the CUDA kernels of ``libhc_gb300.so``; this
package only marshals arguments through its C ABI (``include/hc.h``).  PyTorch
supplies device memory (the workspace) and the CUDA stream.  There is no CPU
fallback: if the library is missing, importing the binding raises.
"""
from ._binding import (  # noqa: F401
    HC_EINVAL, HC_ENOCONV, HC_ENOMEM, HC_ENONFINITE, HC_ENOTSUP, HC_ECUDA, HC_ETIMEOUT,
    HC_EBOUNDS, CHECKED,
    HC_FP32_REFINED, HC_FP32_REFINED_DF, HC_FP64_PLAIN, HC_OK, HC_STOP_DELTA_M, HC_STOP_ENERGY,
    HC_STOP_NONE, HC_STOP_STATUS, HC_PRECOND_SCALAR, HC_PRECOND_KBAR, HuCaiError, Solver,
    StepStats, Batch, hucai_steps, lib, library_path, fp64_fma_peak,
)
