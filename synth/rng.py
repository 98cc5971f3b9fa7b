"""Counter-based splitmix64 draws for the seeded synthetic right-hand sides.

splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; public-domain reference by Vigna) is used as a pure
function of (seed, counter): output i is the finaliser applied to
seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64), which equals the i-th output of
the sequential generator started from state `seed`.

This module holds no arithmetic of the multigrid method; it only produces the
random numbers that both the CUDA path and the oracle receive as inputs.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+n-1 of splitmix64 seeded with `seed` (uint64)."""
    with np.errstate(over="ignore"):
        ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + ctr * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """n i.i.d. uniform[-1, 1) doubles: u = (x >> 11) * 2^-53 * 2 - 1."""
    z = splitmix64(seed, n)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def uniform01(seed: int, n: int) -> np.ndarray:
    """n i.i.d. uniform[0, 1) doubles: u = (x >> 11) * 2^-53."""
    z = splitmix64(seed, n)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def exponential(seed: int, n: int, rate: float) -> np.ndarray:
    """n exponential(rate) inter-arrival gaps by inversion of the 53-bit uniform."""
    z = splitmix64(seed, n)
    u = ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    return -np.log(u) / rate
