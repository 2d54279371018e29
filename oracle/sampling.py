"""Row/column sampling for the linear-scaling ID (Sec. 2.1; oracle, test infrastructure only).

The ID of a tall block A (m >> n) is computed from t*k selected rows A_{s,:} (Eq. pivotedQR2).
The paper allows uniform random rows or rows on a Mock-Chebyshev grid, and prefers the latter
(Sec. 2.1 and Example 1), but does not spell the Mock-Chebyshev grid out. Reading adopted here:
  * Chebyshev nodes of the first kind on [0, 1], t_j = (1 - cos((2j+1) pi / (2s))) / 2 for
    j = 0..s-1, are mapped affinely onto [min C, max C] of the candidates' coordinates;
  * for each node in increasing order, the nearest not-yet-chosen candidate is taken
    (a tie goes to the lower candidate);
  * if there are no more candidates than samples, all candidates are taken;
  * the chosen set is returned in increasing candidate order.
Random sampling draws s distinct candidates by a partial Fisher-Yates shuffle driven by the
SplitMix64 generator (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used as a counter-based generator: draw i of stream `key` is
splitmix64_mix(key + (i + 1) * 0x9E3779B97F4A7C15).
"""
from __future__ import annotations

import math

import numpy as np

_M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64_mix(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def stream_key(seed: int, side: int, step: int, node: int) -> int:
    """Key of the random stream of one ID: side 0 = row IDs (U), 1 = column IDs (V)."""
    return splitmix64_mix(splitmix64_mix(seed) ^ (side << 56) ^ (step << 40) ^ node)


def random_sample(n: int, s: int, key: int):
    if n <= s:
        return np.arange(n)
    swapped = {}
    out = []
    for i in range(s):
        r = splitmix64_mix(key + (i + 1) * GOLDEN)
        j = i + r % (n - i)
        vi, vj = swapped.get(i, i), swapped.get(j, j)
        swapped[j] = vi
        swapped[i] = vj
        out.append(vj)
    return np.sort(np.asarray(out, dtype=np.int64))


def chebyshev_nodes(s: int):
    j = np.arange(s, dtype=np.float64)
    return (1.0 - np.cos((2 * j + 1) * math.pi / (2 * s))) / 2.0


def mock_chebyshev(coords, s: int):
    """Indices (into the ascending array `coords`) of the Mock-Chebyshev sample of size s."""
    c = np.asarray(coords, dtype=np.float64)
    n = c.size
    if n <= s:
        return np.arange(n)
    lo, hi = c[0], c[-1]
    used = np.zeros(n, dtype=bool)
    out = []
    for t in chebyshev_nodes(s):
        y = lo + t * (hi - lo)
        pos = int(np.searchsorted(c, y))
        left = pos - 1
        while left >= 0 and used[left]:
            left -= 1
        right = pos
        while right < n and used[right]:
            right += 1
        if left < 0:
            pick = right
        elif right >= n:
            pick = left
        else:
            pick = left if (y - c[left]) <= (c[right] - y) else right
        used[pick] = True
        out.append(pick)
    return np.sort(np.asarray(out, dtype=np.int64))
