"""Seeded synthetic inputs shared by the oracle pins and the GPU parity tests.

Only random numbers and shapes live here: no step of the method.  Every
generator takes an explicit seed.
"""
import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def real_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """i.i.d. uniform real field in [lo, hi)."""
    return rng(seed).uniform(lo, hi, size=shape)


def complex_array(shape, seed: int) -> np.ndarray:
    g = rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def uint32_counters(n: int, seed: int) -> np.ndarray:
    """n random Philox counters, uint32[n, 4]."""
    return rng(seed).integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)


def uint32_keys(n: int, seed: int) -> np.ndarray:
    return rng(seed).integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
