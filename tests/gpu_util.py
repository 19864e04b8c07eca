"""Helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np


def tol64(values_oracle, scales, rel=1e-12):
    """FP64-path tolerance: rel * max(|f|, S) with S the oracle's condition
    scale (sum of magnitudes of the added pieces)."""
    return rel * np.maximum(np.abs(values_oracle), scales)


def to_dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()
