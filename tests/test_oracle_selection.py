"""Pins for the oracle's community statistics and front selection criteria
(Alg. 3 and the alternatives of Sec. 4.4) (not gpu)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synth


def _brute_stats(rp, ci, lab):
    """Plain definitions with Python integers: communities, sum of squared
    sizes, conductance phi_c = cut_c / min(vol_c, 2m - vol_c) (0 without a
    cut), mean = correctly rounded exact sum (math.fsum) / k, max."""
    n = rp.size - 1
    two_m = int(rp[-1])
    size, vol, cut = {}, {}, {}
    for v in range(n):
        c = int(lab[v])
        size[c] = size.get(c, 0) + 1
        vol[c] = vol.get(c, 0) + int(rp[v + 1] - rp[v])
        cut[c] = cut.get(c, 0) + sum(int(lab[u]) != c for u in ci[rp[v]:rp[v + 1]])
    phis = [cut[c] / min(vol[c], two_m - vol[c]) if cut[c] else 0.0 for c in sorted(size)]
    k = len(size)
    return k, sum(s * s for s in size.values()), math.fsum(phis) / k, max(phis)


def _graphs():
    yield "planted", synth.planted_partition(4, 30, 0.3, 0.03, seed=3)[:2]
    rng = np.random.default_rng(9)
    n = 80
    rp, ci = synth.csr_from_edges(n, rng.integers(0, 70, 300), rng.integers(0, 70, 300))  # 70..79 isolated
    yield "isolated", (rp, ci)
    yield "pair", synth.csr_from_edges(2, [0], [1])


@pytest.mark.parametrize("gi", range(3))
def test_community_stats_brute_force(oracle, gi):
    name, (rp, ci) = list(_graphs())[gi]
    n = rp.size - 1
    labs = [np.zeros(n, np.int32), np.arange(n, dtype=np.int32), (np.arange(n) % 3).astype(np.int32)]
    labs += list(synth.random_labels(n, 6, seed=gi, n_distinct=max(2, n // 4)))
    labs += list(synth.random_labels(n, 3, seed=gi + 10))
    L = np.stack(labs)
    k, sq, mean, mx = oracle.community_stats(rp, ci, L)
    for i in range(L.shape[0]):
        bk, bsq, bmean, bmx = _brute_stats(rp, ci, L[i])
        assert (k[i], sq[i]) == (bk, bsq), (name, i)
        assert mean[i] == bmean and mx[i] == bmx, (name, i)


def test_two_cliques_closed_form(oracle):
    """Two 4-cliques joined by one edge, split along the bridge: vol = 13 on
    each side of 2m = 26, one cut edge, so phi = 1/13 for both communities."""
    u, v = [], []
    for base in (0, 4):
        for a in range(4):
            for b in range(a + 1, 4):
                u.append(base + a)
                v.append(base + b)
    u.append(3)
    v.append(4)
    rp, ci = synth.csr_from_edges(8, u, v)
    k, sq, mean, mx = oracle.community_stats(rp, ci, np.array([0, 0, 0, 0, 1, 1, 1, 1]))
    assert (k[0], sq[0]) == (2, 32)
    assert mean[0] == 1 / 13 and mx[0] == 1 / 13
    # singletons: every non-isolated node has phi = deg / min(deg, 26 - deg) = 1
    k, sq, mean, mx = oracle.community_stats(rp, ci, np.arange(8))
    assert (k[0], sq[0], mean[0], mx[0]) == (8, 8, 1.0, 1.0)
    # one community: no cut anywhere
    k, sq, mean, mx = oracle.community_stats(rp, ci, np.zeros(8, np.int32))
    assert (k[0], sq[0], mean[0], mx[0]) == (1, 64, 0.0, 0.0)


def _brute_select(m, n, k1, k2, stats, criterion, target):
    k, sq, mean, mx = stats

    def key(a):
        if criterion == 1:
            c = abs(int(k[a]) - target)
        elif criterion == 2:
            c = Fraction(int(sq[a]), int(k[a])) - Fraction(n, int(k[a])) ** 2
        elif criterion == 3:
            c = mean[a]
        elif criterion == 4:
            c = mx[a]
        else:
            c = 0
        return (c, 4 * m * int(k1[a]) + int(k2[a]), a)

    return min(range(len(k1)), key=key)


def test_select_solution_brute_force(oracle):
    """Random fronts with many ties in every criterion and in Q."""
    rng = np.random.default_rng(1)
    m, n = 500, 1000
    for trial in range(300):
        cnt = int(rng.integers(1, 40))
        k1 = rng.integers(0, 4, cnt).astype(np.int64) * 10
        k2 = rng.integers(0, 3, cnt).astype(np.int64) * 7
        k = rng.integers(1, 6, cnt).astype(np.int64) * 3
        # sums of squares consistent with k communities over n nodes: >= n^2 / k
        sq = (n * n + k - 1) // k + rng.integers(0, 3, cnt).astype(np.int64) * 1000
        mean = rng.integers(0, 4, cnt) / 8.0
        mx = rng.integers(0, 4, cnt) / 4.0
        stats = (k, sq, mean, mx)
        for criterion in range(5):
            for target in (1, 9, 14):
                got = oracle.select_solution(m, n, k1, k2, stats, criterion, target)
                assert got == _brute_select(m, n, k1, k2, stats, criterion, target), (trial, criterion)


def test_select_variance_exact_near_ties(oracle):
    """Two size variances near 4115 that differ by 3e-7, with n = 2^29: at
    k = 3 the double evaluation of sumsq / k - (n / k)^2 subtracts two values
    near 3.2e16 whose spacing is 4 and orders this pair the wrong way round;
    the exact comparison does not."""
    n = 1 << 29
    ka, kb = 3, (1 << 20) + 1
    sa = (n * n) // ka + 12345
    # pick sb so that var_b is just above var_a: var = (k sq - n^2) / k^2
    num_a = ka * sa - n * n
    target = Fraction(num_a, ka * ka)
    sb = int((target * kb * kb + n * n) / kb) + 1
    assert Fraction(kb * sb - n * n, kb * kb) > target
    stats = (np.array([kb, ka]), np.array([sb, sa]), np.zeros(2), np.zeros(2))
    k1 = np.zeros(2, np.int64)
    k2 = np.zeros(2, np.int64)
    assert oracle.select_solution(1, n, k1, k2, stats, 2, 0) == 1
    stats = (np.array([ka, kb]), np.array([sa, sb]), np.zeros(2), np.zeros(2))
    assert oracle.select_solution(1, n, k1, k2, stats, 2, 0) == 0


def test_select_modularity_is_alg3_best(oracle):
    rp, ci, _ = synth.workload("planted-1k", seed=0)
    p = oracle.Params(pop_size=40, seed=4)
    st = oracle.run(rp, ci, p, oracle.population_init(rp, ci, p), 5)
    m, n = int(rp[-1] // 2), rp.size - 1
    members, best = oracle.pareto_front(st, m)
    stats = oracle.community_stats(rp, ci, st.labels[members])
    assert oracle.select_solution(m, n, st.k1[members], st.k2[members], stats, 0) == best
