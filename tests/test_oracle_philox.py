"""Pins for the oracle's random stream primitives (not gpu).

Philox4x32-10 is checked against the published known-answer vectors of
Salmon et al. (SC'11); the integer pick floor(u k / 2^32) and the coin
thresholds floor(p 2^32) against their exact integer boundaries.
"""
import numpy as np
import pytest

from _golden import GOLDEN

pytestmark = []


def _kat():
    rows = []
    with open(f"{GOLDEN}/philox4x32_10_kat.txt") as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            lhs, rhs = line.split("->")
            a = [int(x, 16) for x in lhs.split()]
            b = [int(x, 16) for x in rhs.split()]
            rows.append((a[:4], a[4:], b))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(oracle, ctr, key, expect):
    assert list(oracle.philox(ctr, key)) == expect


def test_philox_words_are_uniform(oracle):
    # 4 * 8192 words into 64 equal bins: chi-square with 63 dof.
    words = np.concatenate([oracle.philox([c, 7, 3, 2], [11, 13]) for c in range(8192)])
    counts = np.bincount(words >> np.uint32(26), minlength=64)
    exp = words.size / 64
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 110.0  # p < 1e-4 for 63 dof


def test_philox_counter_and_key_change_every_word(oracle):
    base = oracle.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert np.all(oracle.philox(c, [5, 6]) != base)
    assert np.all(oracle.philox([1, 2, 3, 4], [5, 7]) != base)


@pytest.mark.parametrize("k", [1, 2, 3, 7, 100, 1000, 40_000, 1_000_000, (1 << 31) + 5])
def test_pick_boundaries(oracle, k):
    # Index j receives exactly the u with ceil(j 2^32 / k) <= u < ceil((j+1) 2^32 / k).
    two32 = 1 << 32
    for j in sorted({j for j in (0, 1, k // 2, k - 1) if j < k}):
        lo = -(-j * two32 // k)
        assert oracle.pick(lo, k) == j
        if lo > 0:
            assert oracle.pick(lo - 1, k) == j - 1
    assert oracle.pick(two32 - 1, k) == k - 1
    assert oracle.pick(0, k) == 0


def test_thresholds(oracle):
    assert oracle.threshold(0.0) == 0
    assert oracle.threshold(1.0) == 1 << 32
    assert oracle.threshold(0.5) == 1 << 31
    assert oracle.threshold(0.2) == 858993459   # floor(0.2 * 2^32) = floor(858993459.2)
    assert oracle.threshold(0.8) == 3435973836  # floor(3435973836.8)
