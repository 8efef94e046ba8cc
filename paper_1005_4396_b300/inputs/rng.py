"""SplitMix64 counter-based random numbers (Steele, Lea and Flood, OOPSLA 2014).

Every random draw the workloads need (fluence batches, intensities, test
directions, plan parameters) comes from here, so the oracle and the CUDA path
receive identical inputs.  Draw n of stream `seed` is mix(seed + (n+1)*G),
G = 0x9E3779B97F4A7C15, which is what SplitMix64's sequential form yields for
its n-th call after being seeded with `seed`.
"""
import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset..offset+n-1 of the SplitMix64 sequence seeded with `seed`."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _G
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each draw times 2^-53."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals by the Box-Muller transform on consecutive uniform pairs."""
    u = uniform(seed, 2 * n, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
