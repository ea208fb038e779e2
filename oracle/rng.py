"""SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), written as a counter-based generator.

The multigrid setup draws one random start vector per relaxed level for the
Arnoldi eigenvalue estimate (Sec. 4: Chebyshev damping from an estimate of the
largest eigenvalue of M^{-1} K).  Because the oracle and the CUDA library number
DoFs differently, the draw is a pure function of (seed, stream, index):

    z   = seed + (stream * 2^32 + index + 1) * 0x9E3779B97F4A7C15   (mod 2^64)
    z   = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z   = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out = z ^ (z >> 31)

which is the (index+1)-th output of SplitMix64 started at state
seed + stream * 2^32 * gamma.  The value in [-1, 1) is
((out >> 11) * 2^-53) * 2 - 1.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, stream: int, index) -> np.ndarray:
    """Raw 64-bit outputs for an array of indices (uint64 wrap-around)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = np.uint64(stream) * np.uint64(1 << 32) + idx + np.uint64(1)
        z = np.uint64(seed) + ctr * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, stream: int, index) -> np.ndarray:
    """U[-1, 1) doubles from the top 53 bits of the SplitMix64 output."""
    z = splitmix64(seed, stream, index)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0
