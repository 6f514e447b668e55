"""SplitMix64 counter generator for the random initial block X0.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper chooses the initial approximations "randomly" (Section 4.1) and its
drivers take a ``-seed`` flag (Appendix B).  The reading used here: entry
X0[p + n*j] (column-major, point p, column j) is the (p + n*j)-th output
(0-based) of a SplitMix64 generator whose state starts at ``seed``:

    state_i = seed + (i + 1) * 0x9E3779B97F4A7C15          (mod 2**64)
    z = state_i
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9                (mod 2**64)
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB                (mod 2**64)
    out_i = z ^ (z >> 31)

(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014; the constants are Vigna's published SplitMix64 variant), mapped to
[-1, 1) by  2 * (out_i >> 11) * 2**-53 - 1, which is exact in float64.

Pinned by: the published seed-0 output sequence (tests/golden/splitmix64_seed0.txt).
"""

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count, start=0):
    """Outputs ``start .. start+count-1`` of SplitMix64 seeded with ``seed`` (uint64 array)."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_block(seed, n, m):
    """Column-major n-by-m block with entries uniform on [-1, 1) (float64, shape (n, m))."""
    u = splitmix64(seed, n * m)
    x = (u >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    flat = 2.0 * x - 1.0
    # flat index i = p + n*j  ->  column j holds flat[j*n:(j+1)*n]
    return np.ascontiguousarray(flat.reshape(m, n).T)
