"""Pins for the oracle's crossover, mutation, tournament and init (not gpu)."""
from collections import Counter
from itertools import product

import numpy as np
import pytest

import synth
from _golden import graph, ints, load


def test_appendix_e_crossover_and_mutation(oracle):
    """App. E: majority vote of the three drawn parents gives (d); mutating
    node 4 (neighbours {1, 2, 3, 5} = {B, B, B, G}) gives (e)."""
    d = load("appE_operator_example.txt")
    rp, ci = graph(d)
    n = rp.size - 1
    parents = np.stack([ints(d["parent1"]), ints(d["parent2"]), ints(d["parent3"])])
    sel = np.zeros(n, np.uint8)
    sel[int(d["mutate"]) - 1] = 1
    for word in (0, 0x7FFFFFFF, 0xFFFFFFFF):  # no ties arise: any tie word works
        child, q = oracle.operators_forced(rp, ci, parents, np.full(n, word), sel, np.full(n, word))
        assert np.array_equal(child, ints(d["child"]))
        assert np.array_equal(q, ints(d["mutated"]))


def test_mode_pick_brute_force(oracle):
    """Every multiset of up to 5 labels from {0..3}: the result is the
    pick(u, t)-th smallest of the t most frequent labels (Eq. arg_max)."""
    for k in range(1, 6):
        for xs in product(range(4), repeat=k):
            cnt = Counter(xs)
            top = max(cnt.values())
            ties = sorted(c for c, v in cnt.items() if v == top)
            for u in (0, 0x40000000, 0x80000000, 0xC0000000, 0xFFFFFFFF):
                j = (u * len(ties)) >> 32
                assert oracle.mode_pick(np.array(xs), u) == ties[j]


def test_tie_break_is_uniform(oracle):
    xs = np.array([9, 3, 5, 7, 3, 5, 7, 9], np.int32)  # four labels tied at 2
    rng = np.random.default_rng(0)
    got = Counter(oracle.mode_pick(xs, int(u)) for u in rng.integers(0, 1 << 32, 4000))
    assert set(got) == {3, 5, 7, 9}
    chi2 = sum((v - 1000) ** 2 / 1000 for v in got.values())
    assert chi2 < 21.1  # 3 dof, p < 1e-4


def test_tournament_winner_distribution(oracle):
    """Binary tournament on P sorted by (rank, crowding): the winner is sorted
    position min(a, b), so P(position s) = (2 (N - s) - 1) / N^2."""
    Np = 20
    params = oracle.Params(pop_size=Np, n_parents=4, seed=123)
    # Keys on a dominance chain: individual p has rank p' where p' = perm[p].
    perm = np.random.default_rng(1).permutation(Np)
    k1 = perm.astype(np.int64)
    k2 = perm.astype(np.int64)
    counts = np.zeros(Np)
    xo_total = 0
    for gen in range(1, 401):
        par, xo, skip = oracle.select_parents(params, gen, k1, k2)
        counts += np.bincount(perm[par.ravel()], minlength=Np)
        xo_total += xo.sum()
        assert np.all((skip >= 0) & (skip < 4))
    total = counts.sum()
    s = np.arange(Np)
    exp = total * (2 * (Np - s) - 1) / Np ** 2
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 50.0  # 19 dof, p < 1e-4
    frac = xo_total / (400 * Np)
    assert abs(frac - 0.8) < 0.03  # crossover coin ~ C_P


def test_init_population_uniform_labels(oracle):
    n = 257
    P = oracle.init_population(n, oracle.Params(pop_size=64, seed=5))
    assert P.min() >= 0 and P.max() < n
    counts = np.bincount(P.ravel(), minlength=n)
    exp = P.size / n
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 256 + 6 * np.sqrt(2 * 256)
    assert not np.array_equal(P[0], P[1])


def test_offspring_labels_and_mutation_rate(oracle):
    rp, ci, _ = synth.planted_partition(4, 40, 0.3, 0.02, seed=2)
    n = rp.size - 1
    params = oracle.Params(pop_size=16, seed=9, p_crossover=1.0, p_mutation=0.2)
    st = oracle.population_init(rp, ci, params)
    Q, qk1, qk2 = oracle.make_offspring(rp, ci, params, 1, st)
    assert Q.min() >= 0 and Q.max() < n
    intra, S = oracle.objectives(rp, ci, Q)
    m = rp[-1] // 2
    assert np.array_equal(qk1, m - intra) and np.array_equal(qk2, S)
    # With C_P = 0 and M_P = 0 every child is a copy of one of its parents.
    p0 = oracle.Params(pop_size=16, seed=9, p_crossover=0.0, p_mutation=0.0)
    Q0, _, _ = oracle.make_offspring(rp, ci, p0, 1, st)
    par, xo, skip = oracle.select_parents(p0, 1, st.k1, st.k2)
    for i in range(16):
        if not xo[i]:
            assert np.array_equal(Q0[i], st.labels[par[i, skip[i]]])
    # With M_P = 1 every node of positive degree takes a neighbour's label.
    p1 = oracle.Params(pop_size=16, seed=9, p_crossover=0.0, p_mutation=1.0)
    Q1, _, _ = oracle.make_offspring(rp, ci, p1, 1, st)
    deg = np.diff(rp)
    for i in range(4):
        for v in range(n):
            if deg[v]:
                assert Q1[i, v] in set(st.labels[par[i, skip[i]]][ci[rp[v]:rp[v + 1]]].tolist())


def _sweep_graph():
    """Small graph with a hub, a path, isolated nodes and adjacency rows given
    in shuffled order (the oracle may not rely on sorted rows)."""
    rng = np.random.default_rng(17)
    n = 60
    u = list(rng.integers(0, 50, 120)) + [50] * 8 + [51, 52]
    v = list(rng.integers(0, 50, 120)) + list(range(40, 48)) + [52, 53]
    rp, ci = synth.csr_from_edges(n, u, v)  # nodes 54..59 isolated
    for a in range(n):
        seg = ci[rp[a]:rp[a + 1]].copy()
        rng.shuffle(seg)
        ci[rp[a]:rp[a + 1]] = seg
    return rp, ci


@pytest.mark.parametrize("seed", [0, 13, (1 << 40) + 5])
def test_init_sweep_closed_form(oracle, seed):
    """init_mode 1 = singletons, then one synchronous full-rate neighbour
    majority step. Singleton labels are the node ids, all distinct, so every
    neighbour of v ties at count 1 and the step takes the pick(u, deg v)-th
    smallest neighbour id, u the INIT word of (v, i); degree 0 keeps v."""
    rp, ci = _sweep_graph()
    n = rp.size - 1
    Np = 11
    st = oracle.population_init(rp, ci, oracle.Params(pop_size=Np, seed=seed, init_mode=1))
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in range(Np):
        for v in range(n):
            nb = sorted(ci[rp[v]:rp[v + 1]].tolist())
            if not nb:
                assert st.labels[i, v] == v
                continue
            u = int(oracle.philox((v, i // 4, 0, 1), key)[i % 4])
            assert st.labels[i, v] == nb[(u * len(nb)) >> 32]
    intra, S = oracle.objectives(rp, ci, st.labels)
    m = int(rp[-1] // 2)
    assert np.array_equal(st.k1, m - intra) and np.array_equal(st.k2, S)


def test_init_sweep_two_node_path_and_isolated(oracle):
    """0 - 1, 2 isolated: the synchronous step swaps the labels of 0 and 1
    (each sees only the other's singleton label), node 2 keeps label 2."""
    rp, ci = synth.csr_from_edges(3, [0], [1])
    st = oracle.population_init(rp, ci, oracle.Params(pop_size=5, seed=2, init_mode=1))
    assert np.array_equal(st.labels, np.tile([1, 0, 2], (5, 1)))
    assert np.all(st.k1 == 1) and np.all(st.k2 == 2)  # intra 0; D = 1, 1


# ---------------------------------------------------------------------------
# The random-stream operators that every run uses (crossover_child,
# mutate_child and the skip-branch parent of orc_make_offspring_range),
# re-derived here by brute force: Counter majorities in plain Python, the
# tournament from the rank/crowding order (pinned in test_oracle_nsga.py),
# every random word recomputed from Philox (pinned by the published test
# vectors) with the stream layout written out below, independently of the
# oracle's own helpers.
# ---------------------------------------------------------------------------

ST_SELECT, ST_XTIE, ST_MCOIN, ST_MTIE = 2, 3, 4, 5


def _node_word(oracle, key, stage, gen, i, v):
    """Word of (individual i, node v): counter (v, i // 4, gen, stage), word i % 4."""
    return int(oracle.philox((v, i // 4, gen, stage), key)[i % 4])


def _select_word(oracle, key, gen, i, w):
    """Selection word w of child i: counter (w // 4, i, gen, 2), word w % 4."""
    return int(oracle.philox((w // 4, i, gen, ST_SELECT), key)[w % 4])


def _pick(u, k):
    return (u * k) >> 32


def _majority(values, u):
    """Most frequent value; among the t tied ones (ascending) the pick(u, t)-th."""
    cnt = Counter(values)
    top = max(cnt.values())
    ties = sorted(c for c, k in cnt.items() if k == top)
    return ties[_pick(u, len(ties))] if len(ties) > 1 else ties[0]


def _brute_offspring(oracle, rp, ci, params, gen, P, k1, k2):
    """Q of generation `gen` (Alg. 1 parallel map: tournament, Alg. 2
    crossover, Sec. 4.3.2 mutation) written out node by node."""
    Np, E, n = params.pop_size, params.n_parents, rp.size - 1
    key = (params.seed & 0xFFFFFFFF, params.seed >> 32)
    thr_c = int(np.floor(params.p_crossover * 2.0 ** 32))
    thr_m = int(np.floor(params.p_mutation * 2.0 ** 32))
    _, _, order = oracle.rank_crowd_order(k1, k2)
    Q = np.zeros((Np, n), np.int32)
    parents, crossed, skipped = [], [], []
    for i in range(Np):
        par = []
        for j in range(E):
            a = _pick(_select_word(oracle, key, gen, i, 2 * j), Np)
            b = _pick(_select_word(oracle, key, gen, i, 2 * j + 1), Np)
            par.append(int(order[min(a, b)]))  # binary tournament on the sorted P
        cross = _select_word(oracle, key, gen, i, 2 * E) <= thr_c
        skip = _pick(_select_word(oracle, key, gen, i, 2 * E + 1), E)
        parents.append(par)
        crossed.append(cross)
        skipped.append(skip)
        if cross:
            child = [
                _majority([int(P[p, v]) for p in par], _node_word(oracle, key, ST_XTIE, gen, i, v))
                for v in range(n)]
        else:
            child = [int(x) for x in P[par[skip]]]
        for v in range(n):
            nb = ci[rp[v]:rp[v + 1]]
            Q[i, v] = child[v]
            if nb.size and _node_word(oracle, key, ST_MCOIN, gen, i, v) < thr_m:
                Q[i, v] = _majority([child[u] for u in nb], _node_word(oracle, key, ST_MTIE, gen, i, v))
    return Q, np.array(parents), np.array(crossed), np.array(skipped)


def _operator_graph():
    """Two dense communities, a hub of degree 30, a path, isolated nodes."""
    rng = np.random.default_rng(5)
    n = 96
    u, v = [], []
    for base in (0, 30):
        a = rng.integers(base, base + 30, 160)
        b = rng.integers(base, base + 30, 160)
        u += list(a)
        v += list(b)
    u += [60] * 30
    v += list(range(61, 91))
    u += [91, 92]
    v += [92, 93]  # path 91 - 92 - 93; nodes 94, 95 isolated
    return synth.csr_from_edges(n, u, v)


@pytest.mark.parametrize("cp,mp,seed,alphabet", [
    (1.0, 0.0, 0, 3),            # crossover only: every node is a vote of E_S parents
    (0.0, 1.0, 7, 3),            # copy branch, then mutation of every node
    (0.8, 0.2, (1 << 40) + 3, 4),  # the paper's rates, both key words non-zero
    (0.8, 0.5, 11, 2),           # two labels: ties at every even degree
])
def test_offspring_brute_force(oracle, cp, mp, seed, alphabet):
    """Every child of two consecutive generations equals the brute-force
    tournament -> majority crossover (or copy of the skip-branch parent) ->
    neighbour-majority mutation, with the labels drawn from a small alphabet
    so that ties (and hence the tie words) decide many nodes."""
    rp, ci = _operator_graph()
    n = rp.size - 1
    m = int(rp[-1] // 2)
    params = oracle.Params(pop_size=12, n_parents=4, p_crossover=cp, p_mutation=mp, seed=seed)
    rng = np.random.default_rng(seed & 0xFFFF)
    ids = rng.choice(n, alphabet, replace=False)
    P = ids[rng.integers(0, alphabet, (params.pop_size, n))].astype(np.int32)
    intra, S = oracle.objectives(rp, ci, P)
    st = oracle.State(P, m - intra, S, 0)
    for gen in (1, 2):
        Q, qk1, qk2 = oracle.make_offspring(rp, ci, params, gen, st)
        want, par, crossed, skip = _brute_offspring(oracle, rp, ci, params, gen, st.labels, st.k1, st.k2)
        opar, oxo, oskip = oracle.select_parents(params, gen, st.k1, st.k2)
        assert np.array_equal(opar, par), "tournament parents differ"
        assert np.array_equal(oxo.astype(bool), crossed), "crossover coins differ"
        assert np.array_equal(oskip, skip), "skip-branch parent differs"
        assert np.array_equal(Q, want), "offspring differ from the brute-force operators"
        i2, s2 = oracle.objectives(rp, ci, Q)
        assert np.array_equal(qk1, m - i2) and np.array_equal(qk2, s2)
        if cp == 1.0:
            assert crossed.all()
        if cp == 0.0:
            assert not crossed.any()
        st = oracle.run(rp, ci, params, st, 1)


def test_mutation_takes_the_majority_not_any_neighbour(oracle):
    """A node whose neighbours hold labels {a, a, a, b} must take a under
    mutation at rate 1 (a random neighbour label would give b a quarter of
    the time): the hub 0 with neighbours 1..4, all copies of one parent."""
    rp, ci = synth.csr_from_edges(5, [0, 0, 0, 0], [1, 2, 3, 4])
    params = oracle.Params(pop_size=40, n_parents=2, p_crossover=0.0, p_mutation=1.0, seed=3)
    P = np.tile(np.array([4, 2, 2, 2, 3], np.int32), (params.pop_size, 1))
    intra, S = oracle.objectives(rp, ci, P)
    st = oracle.State(P, 4 - intra, S, 0)
    Q, _, _ = oracle.make_offspring(rp, ci, params, 1, st)
    assert np.all(Q[:, 0] == 2)        # neighbours 2, 2, 2, 3
    assert np.all(Q[:, 1:] == 4)       # each leaf sees only the hub's label 4
