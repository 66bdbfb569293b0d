"""Pins for the oracle's non-dominated sort, crowding and selection (not gpu).

The sort is checked against the Pareto front of *every* partition of small
graphs (brute force over all set partitions, Sec. 2.2 definitions) and against
an independent characterisation of Deb's ranks: rank(p) is one more than the
largest rank among the points dominating p.
"""
import numpy as np
import pytest

import synth
from _golden import graph, load


def _set_partitions(n):
    """All set partitions of n items as restricted-growth label vectors."""
    out = []
    a = [0] * n

    def rec(i, mx):
        if i == n:
            out.append(list(a))
            return
        for c in range(mx + 2):
            a[i] = c
            rec(i + 1, max(mx, c))
    a[0] = 0
    rec(1, 0)
    return np.array(out, dtype=np.int32)


def _dominates(k1, k2):
    """dom[q, p] = q dominates p."""
    a1, a2 = k1[:, None], k2[:, None]
    b1, b2 = k1[None, :], k2[None, :]
    return (a1 <= b1) & (a2 <= b2) & ((a1 < b1) | (a2 < b2))


def _chain_rank(k1, k2):
    order = np.lexsort((k2, k1))  # a dominator is lexicographically smaller
    rank = np.zeros(k1.size, dtype=np.int64)
    for p in order:
        dom = (k1 <= k1[p]) & (k2 <= k2[p]) & ((k1 < k1[p]) | (k2 < k2[p]))
        rank[p] = 1 + (rank[dom].max() if dom.any() else 0)
    return rank


def test_bell_numbers():
    assert [len(_set_partitions(n)) for n in range(1, 9)] == [1, 2, 5, 15, 52, 203, 877, 4140]


@pytest.mark.parametrize("case", ["appE", "random7"])
def test_front_equals_brute_force_pareto_front(oracle, case):
    if case == "appE":
        rp, ci = graph(load("appE_operator_example.txt"))
    else:
        rng = np.random.default_rng(11)
        iu, ju = np.triu_indices(7, 1)
        keep = rng.random(iu.size) < 0.45
        rp, ci = synth.csr_from_edges(7, iu[keep], ju[keep])
    n = rp.size - 1
    m = int(rp[-1] // 2)
    parts = _set_partitions(n)
    intra, S = oracle.objectives(rp, ci, parts)
    k1, k2 = m - intra, S
    dom = _dominates(k1, k2)
    pf = ~dom.any(axis=0)  # Sec. 2.2: no point dominates p
    rank = oracle.nondominated_sort(k1, k2)
    assert np.array_equal(rank == 1, pf)
    assert np.array_equal(rank, _chain_rank(k1, k2))


def test_rank_matches_chain_rank_with_ties(oracle):
    rng = np.random.default_rng(2)
    for trial in range(20):
        N = int(rng.integers(1, 220))
        k1 = rng.integers(0, 12, N).astype(np.int64)
        k2 = rng.integers(0, 12, N).astype(np.int64)
        rank = oracle.nondominated_sort(k1, k2)
        assert np.array_equal(rank, _chain_rank(k1, k2))
        dom = _dominates(k1, k2)
        for p in range(N):
            same = rank == rank[p]
            assert not dom[same, p].any()  # no domination inside a front
            if rank[p] > 1:
                assert dom[rank == rank[p] - 1, p].any()


def test_crowding_closed_forms(oracle):
    # Five equally spaced points on a line: each interior neighbour gap is 2/4
    # of the range in both objectives.
    k1 = np.array([0, 1, 2, 3, 4], np.int64)
    k2 = np.array([4, 3, 2, 1, 0], np.int64)
    c = oracle.crowding(k1, k2, np.ones(5, np.int32))
    assert np.isinf(c[0]) and np.isinf(c[4]) and np.all(c[1:4] == 1.0)
    # Uneven front: p1 gets 5/10 + 7/10, p2 gets 9/10 + 8/10.
    k1 = np.array([0, 1, 5, 10], np.int64)
    k2 = np.array([10, 8, 3, 0], np.int64)
    c = oracle.crowding(k1, k2, np.ones(4, np.int32))
    assert np.isinf(c[0]) and np.isinf(c[3])
    assert c[1] == 0.5 + 0.7 and c[2] == 0.9 + 0.8
    # Fronts of one or two members are all +inf.
    c = oracle.crowding(np.array([0, 3, 1], np.int64), np.array([3, 0, 5], np.int64),
                        np.array([1, 1, 2], np.int32))
    assert np.all(np.isinf(c))
    # Identical points: the first and last by position are the ends, the rest 0.
    c = oracle.crowding(np.full(4, 7, np.int64), np.full(4, 9, np.int64), np.ones(4, np.int32))
    assert np.isinf(c[0]) and np.isinf(c[3]) and c[1] == 0.0 and c[2] == 0.0


def test_crowding_is_scale_free_and_positive(oracle):
    rng = np.random.default_rng(5)
    k1 = np.sort(rng.choice(1000, 30, replace=False)).astype(np.int64)
    k2 = np.sort(rng.choice(1000, 30, replace=False))[::-1].astype(np.int64).copy()
    r = np.ones(30, np.int32)
    a = oracle.crowding(k1, k2, r)
    b = oracle.crowding(k1 * 7 + 3, k2 * 5 + 11, r)
    assert np.allclose(a[1:-1], b[1:-1], rtol=1e-15) and np.all(a[1:-1] > 0)


def test_sort_by_rank_and_crowding(oracle):
    rng = np.random.default_rng(6)
    k1 = rng.integers(0, 50, 200).astype(np.int64)
    k2 = rng.integers(0, 50, 200).astype(np.int64)
    rank, crowd, order = oracle.rank_crowd_order(k1, k2)
    assert sorted(order.tolist()) == list(range(200))
    for a, b in zip(order[:-1], order[1:]):
        assert (rank[a], -crowd[a], a) < (rank[b], -crowd[b], b)


def test_environmental_selection(oracle):
    rng = np.random.default_rng(7)
    for _ in range(10):
        rk1 = rng.integers(0, 40, 200).astype(np.int64)
        rk2 = rng.integers(0, 40, 200).astype(np.int64)
        keep = oracle.env_select(rk1, rk2)
        rank, crowd, _ = oracle.rank_crowd_order(rk1, rk2)
        assert len(set(keep.tolist())) == 100
        last = rank[keep].max()
        # Every front before the last one is kept whole ...
        assert np.all(np.isin(np.nonzero(rank < last)[0], keep))
        # ... and the last front keeps its most crowded-apart members.
        kept_last = crowd[keep][rank[keep] == last]
        dropped = np.setdiff1d(np.nonzero(rank == last)[0], keep)
        if dropped.size:
            assert kept_last.min() >= crowd[dropped].max()
        # The kept list is in (rank, crowding desc, index) order.
        for a, b in zip(keep[:-1], keep[1:]):
            assert (rank[a], -crowd[a], a) < (rank[b], -crowd[b], b)
