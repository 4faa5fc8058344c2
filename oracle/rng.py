"""SplitMix64 used as a counter-based generator (oracle side).

Definition (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the i-th output for a stream with seed S is the
64-bit finaliser applied to  z = S + (i + 1) * 0x9E3779B97F4A7C15  (mod 2^64):
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)
A uniform double in [-1, 1) is taken from the top 53 bits:  2 * (z >> 11) * 2^-53 - 1,
which is exact in binary64, so both implementations produce identical vectors.

The method draws random numbers twice: the Lanczos start vector and the block
of starting vectors for the count-to-threshold estimate.  Stream ids keep the
two apart (see ``partial.py``).
"""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the SplitMix64 stream for `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [-1, 1) from the top 53 bits of each SplitMix64 output."""
    z = splitmix64(seed, count, offset)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def gaussian(seed: int, count: int) -> np.ndarray:
    """Standard normal doubles by the Box-Muller transform (Box and Muller, Ann. Math. Stat.
    1958) of consecutive SplitMix64 pairs: output 2j uses cos and output 2j + 1 sin of the
    same pair (u1, u2), with u1 = ((z_{2j} >> 11) + 1) 2^-53 in (0, 1] (so log(u1) is finite)
    and u2 = (z_{2j+1} >> 11) 2^-53 in [0, 1):
        g_{2j}   = sqrt(-2 log u1) cos(2 pi u2)
        g_{2j+1} = sqrt(-2 log u1) sin(2 pi u2)
    The device implements the same definition; the transcendental functions round differently
    there, so the two agree to a few ulps, not bit for bit."""
    pairs = (count + 1) // 2
    z = splitmix64(seed, 2 * pairs)
    u1 = ((z[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (z[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * pairs)
    out[0::2] = r * np.cos(2.0 * np.pi * u2)
    out[1::2] = r * np.sin(2.0 * np.pi * u2)
    return out[:count]
