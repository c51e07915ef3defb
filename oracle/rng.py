"""Counter-based generator of the oracle: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; constants as published by Vigna).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The CUDA library implements the same
published generator independently; it provides the start vector of the CG eigenvalue
estimate (Sec. 3.2.1), whose choice the paper leaves open.

value(seed, level, i) = 2 * (splitmix64(seed + level * 2^40 + i) >> 11) * 2^-53 - 1, in [-1, 1).
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """One SplitMix64 output for each 64-bit counter value x (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, level: int, n: int) -> np.ndarray:
    with np.errstate(over="ignore"):
        key = np.uint64(seed) + np.uint64(level) * np.uint64(1 << 40) + np.arange(n, dtype=np.uint64)
    z = splitmix64(key) >> np.uint64(11)
    return 2.0 * (z.astype(np.float64) * 2.0 ** -53) - 1.0
