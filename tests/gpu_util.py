"""Helpers for the GPU tests (skip cleanly when no CUDA device is present)."""
import numpy as np
import pytest

PAPER = dict(Du=0.2, Dv=0.1, F=0.02, k=0.048, dt=1.0)


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_10292_gb300 import gs
    gs.lib()
    return torch


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))))
