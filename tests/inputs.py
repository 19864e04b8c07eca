"""Seeded synthetic input generators shared by the oracle tests and the GPU
parity tests.  Holds none of the method's arithmetic: it only draws the test
inputs (populations to evaluate, near-optimum offsets), with numpy's PCG64.
"""
import numpy as np


def uniform_pop(N, D, seed=12345, lb=-100.0, ub=100.0):
    """X ~ U[lb, ub]^{N x D} (the batched-evaluation microbench input)."""
    return np.random.default_rng(seed).uniform(lb, ub, size=(N, D))


def near(center, N, scale, seed=7):
    """N points center + scale * N(0, 1): near-optimum probes."""
    rng = np.random.default_rng(seed)
    c = np.asarray(center, dtype=np.float64)
    return c[None, :] + scale * rng.standard_normal((N, c.shape[0]))


def mixed_scales(center, N, D, seed=11):
    """Points at distances spread over 1e-6 .. 1e2 from center."""
    rng = np.random.default_rng(seed)
    c = np.asarray(center, dtype=np.float64)
    dirs = rng.standard_normal((N, D))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = 10.0 ** rng.uniform(-6, 2, size=(N, 1))
    return np.clip(c[None, :] + r * dirs, -100.0, 100.0)
