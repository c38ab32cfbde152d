"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Holds none of the method's arithmetic: only random numbers.  Populations built from them are
w_j (1 + a r) with r ~ U(-1, 1) (seed 0 and 1 by default), assembled by the caller.
"""
import numpy as np


def uniform(seed: int, shape) -> np.ndarray:
    """U(-1, 1) draws in float64 from numpy's PCG64 generator."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape)
