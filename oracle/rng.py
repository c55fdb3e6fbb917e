"""splitmix64 counter-based generator (Steele, Lea, Flood, OOPSLA 2014).

Used only for the Lanczos start vector of the eigenvalue estimate, whose
random draws are internal to the method's setup.  Written from the
generator's published definition; the CUDA library has its own copy.
"""
import numpy as np

_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n values in [-1, 1): state_k = seed + (k+1)*golden, mixed, top 53 bits -> [0,1), then 2u-1."""
    out = np.empty(n, np.float64)
    s = seed & _MASK
    for k in range(n):
        s = (s + _GOLDEN) & _MASK
        z = s
        z = ((z ^ (z >> 30)) * _M1) & _MASK
        z = ((z ^ (z >> 27)) * _M2) & _MASK
        z = z ^ (z >> 31)
        out[k] = 2.0 * ((z >> 11) * (1.0 / 9007199254740992.0)) - 1.0
    return out
