"""Counter-based random numbers: the SplitMix64 generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).

The n-th output (n = 0, 1, ...) of SplitMix64 seeded with `seed` is
mix(seed + (n + 1) * GAMMA) with GAMMA = 0x9E3779B97F4A7C15, where mix is the
generator's finaliser.  Using n as a counter makes every draw addressable by
an index (a cell index, a split number), so inputs never depend on the order
in which they are generated.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, n):
    """n-th SplitMix64 output for `seed` (n: int or integer array)."""
    with np.errstate(over="ignore"):
        n = np.asarray(n, dtype=np.uint64)
        z = np.uint64(seed) + (n + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed, n):
    """Uniform double in [0, 1) from the top 53 bits of the n-th output."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def std_normal(seed, n):
    """Standard normal draws by Box-Muller: draw m uses uniforms 2m, 2m+1."""
    n = np.asarray(n, dtype=np.uint64)
    u1 = 1.0 - uniform01(seed, np.uint64(2) * n)          # (0, 1]
    u2 = uniform01(seed, np.uint64(2) * n + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def subseed(seed, tag):
    """Independent stream seed for a named purpose (tag: small integer)."""
    return int(splitmix64(seed, np.uint64(0xD1B54A32D192ED03) ^ np.uint64(tag)))
