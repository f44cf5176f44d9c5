"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the multigrid method: it only turns
(seed, index) pairs into numbers.  The generator is SplitMix64 (Steele, Lea,
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), used in
counter form: value i of stream `seed` is the SplitMix64 output for the state
seed + (i+1) * 0x9E3779B97F4A7C15.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n consecutive SplitMix64 outputs of stream `seed`, starting at index `offset`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def initial_guess(n: int, seed: int = 1) -> np.ndarray:
    """u0 with entries uniform on [-1, 1] (the paper's random initial guess, Sec. 5)."""
    return 2.0 * uniform01(seed, n) - 1.0


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normal samples by the Box-Muller transform of two uniform streams."""
    u1 = uniform01(seed, n, offset)
    u2 = uniform01(seed ^ 0x5DEECE66D, n, offset)
    u1 = np.maximum(u1, 1e-300)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def batched_rhs(f: np.ndarray, nrhs: int, seed: int = 2, noise: float = 0.01) -> np.ndarray:
    """nrhs right-hand sides: f scaled by a per-RHS factor uniform on [0.5, 2] plus
    nodal noise with standard deviation `noise` * max|f|.  Shape (nrhs, len(f))."""
    out = np.empty((nrhs, f.size))
    scale = 0.5 + 1.5 * uniform01(seed, nrhs)
    amp = noise * float(np.max(np.abs(f))) if f.size else 0.0
    for r in range(nrhs):
        out[r] = scale[r] * f + amp * normal(seed + 1 + r, f.size)
    return out
