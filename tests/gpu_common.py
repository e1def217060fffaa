"""Shared helpers of the GPU parity tests (pure marshalling, no arithmetic of
the scheme)."""
import os

import numpy as np
import pytest


def rel_l2(a, b) -> float:
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


def packed(F: np.ndarray) -> np.ndarray:
    """Packed half-spectrum layout of a full 2D spectrum F[ky, kx]:
    P[:, kx] = F[:, kx] for 1 <= kx < nx/2, P[:, 0] = F[:, 0] + i F[:, nx/2]."""
    ny, nx = F.shape
    H = nx // 2
    P = F[:, :H].copy()
    P[:, 0] = F[:, 0] + 1j * F[:, H]
    return P


@pytest.fixture(scope="session")
def hc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_2606_06720_gb300 as P
    import oracle as O
    O.set_threads(os.cpu_count() or 1)
    return P
