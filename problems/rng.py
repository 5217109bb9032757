"""Counter-based seeded random numbers shared by every consumer of the
synthetic inputs.

The generator is SplitMix64 as published by S. Vigna (the state advances by
the golden-ratio increment 0x9E3779B97F4A7C15 and each output is the
"mix13" finaliser of the new state).  Because the i-th output depends only on
(seed, i), a vector of any length is produced in one vectorised numpy pass.

Nothing here computes any part of the solver method; it only draws numbers.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of SplitMix64 seeded with ``seed``.

    Output i (0-based) is mix(seed + (i+1)*GAMMA) with mix the published
    finaliser; arithmetic wraps modulo 2**64 as in the definition.
    """
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each SplitMix64 output times 2**-53."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, count: int, lo: float, hi: float, offset: int = 0) -> np.ndarray:
    """Doubles in [lo, hi): lo + (hi - lo) * u with u from :func:`uniform01`."""
    return lo + (hi - lo) * uniform01(seed, count, offset)


def x_true(seed: int, n: int) -> np.ndarray:
    """The manufactured solution: n doubles uniform in [-1, 1) (2u - 1)."""
    return 2.0 * uniform01(seed, n) - 1.0
