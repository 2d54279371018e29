"""Pins of the oracle's Mock-Chebyshev and random sampling (Sec. 2.1)."""
import os

import numpy as np
import pytest

from oracle import sampling

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


def test_splitmix64_published_vectors():
    want = [int(v, 16) for v in _read("splitmix64.txt")]
    got = [sampling.splitmix64_mix((i + 1) * sampling.GOLDEN) for i in range(3)]
    assert got == want


def test_mock_chebyshev_worked_example():
    want = [int(v) for v in _read("mock_chebyshev_11_3.txt")]
    assert list(sampling.mock_chebyshev(np.arange(11.0), 3)) == want


def _brute_mock(c, s):
    n = len(c)
    if n <= s:
        return list(range(n))
    t = (1 - np.cos((2 * np.arange(s) + 1) * np.pi / (2 * s))) / 2
    used = set()
    for tj in t:
        y = c[0] + tj * (c[-1] - c[0])
        best = None
        for i in range(n):          # scan every candidate: nearest unused, ties to the lower index
            if i in used:
                continue
            if best is None or abs(c[i] - y) < abs(c[best] - y):
                best = i
        used.add(best)
    return sorted(used)


@pytest.mark.parametrize("n,s,seed", [(50, 7, 1), (40, 39, 2), (300, 64, 3), (20, 20, 4), (9, 12, 5)])
def test_mock_chebyshev_matches_brute_force(n, s, seed):
    rng = np.random.default_rng(seed)
    c = np.sort(rng.uniform(-3, 8, n))
    got = list(sampling.mock_chebyshev(c, s))
    assert got == _brute_mock(c, s)
    assert len(set(got)) == min(n, s)


def test_mock_chebyshev_clusters_at_the_ends():
    got = sampling.mock_chebyshev(np.arange(10000.0), 20)
    gaps = np.diff(got)
    assert gaps[0] < gaps[len(gaps) // 2] and gaps[-1] < gaps[len(gaps) // 2]


def test_random_sample_is_a_seeded_subset():
    a = sampling.random_sample(1000, 50, sampling.stream_key(3, 0, 2, 17))
    b = sampling.random_sample(1000, 50, sampling.stream_key(3, 0, 2, 17))
    c = sampling.random_sample(1000, 50, sampling.stream_key(3, 0, 2, 18))
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert len(set(a.tolist())) == 50 and a.min() >= 0 and a.max() < 1000
    assert np.all(np.diff(a) > 0)
    assert np.array_equal(sampling.random_sample(7, 9, 1), np.arange(7))


def test_random_sample_is_roughly_uniform():
    n, s, trials = 40, 10, 2000
    counts = np.zeros(n)
    for k in range(trials):
        counts[sampling.random_sample(n, s, sampling.stream_key(k, 1, 1, 0))] += 1
    expected = trials * s / n
    chi2 = np.sum((counts - expected) ** 2 / expected)
    assert chi2 < 100  # 39 degrees of freedom; p ~ 1e-6 at this bound
