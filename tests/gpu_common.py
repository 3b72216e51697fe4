"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
import numpy as np


def relerr(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def maxerr(a, b) -> float:
    """max_i |a_i - b_i| / max_i |b_i|"""
    a = np.asarray(a)
    b = np.asarray(b)
    mb = np.abs(b).max()
    return float(np.abs(a - b).max() / (mb if mb > 0 else 1.0))


def cuda_or_fail():
    import torch
    assert torch.cuda.is_available(), "GPU test without a CUDA device"
    return torch
