"""The random shadow vector r~_{-1} with which Alg. 2 starts.

The paper leaves the distribution open.  Both the oracle and the CUDA path
draw it from one counter-based generator, SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014; the 64-bit
finaliser constants are those of Vigna's public reference implementation):

    state_i = seed + (i + 1) * 0x9E3779B97F4A7C15           (mod 2^64)
    z = (state_i ^ (state_i >> 30)) * 0xBF58476D1CE4E5B9      (mod 2^64)
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB                  (mod 2^64)
    out_i = z ^ (z >> 31)

and r~_{-1}[i] = 2 * ((out_i >> 11) * 2^-53) - 1, an exactly representable
double in [-1, 1).  This file is written independently of the CUDA
generator; the two share no code.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1
DEFAULT_SEED = 0x5EED


def splitmix64_scalar(seed: int, i: int) -> int:
    """Output i (0-based) of SplitMix64 started from state ``seed`` (pure Python ints)."""
    z = (seed + (i + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """Outputs 0..n-1 of SplitMix64 from state ``seed`` as uint64 (vectorised)."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + i * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        z = z ^ (z >> np.uint64(31))
    return z


def shadow_vector(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """r~_{-1}: n doubles in [-1, 1) from SplitMix64(seed)."""
    z = splitmix64(seed, n)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0
