"""Whole-run pins for the oracle (not gpu): Alg. 1 recovers a planted
partition, runs are reproducible and resumable, and the front it returns is
non-dominated with the recommended member maximising Q = 1 - f1 - f2."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def planted():
    return synth.workload("planted-1k", seed=0)


@pytest.fixture(scope="module")
def planted_run(oracle, planted):
    rp, ci, _ = planted
    params = oracle.Params(seed=0)
    st0 = oracle.population_init(rp, ci, params)
    return params, st0, oracle.run(rp, ci, params, st0, 100)


def test_planted_partition_recovered(oracle, planted, planted_run):
    sk = pytest.importorskip("sklearn.metrics")
    rp, ci, truth = planted
    _, _, st = planted_run
    m = int(rp[-1] // 2)
    members, best = oracle.pareto_front(st, m)
    lab = st.labels[members[best]]
    nmi = sk.normalized_mutual_info_score(truth, lab)
    assert nmi >= 0.9, nmi


def test_front_and_recommended_solution(oracle, planted, planted_run):
    rp, _, _ = planted
    _, _, st = planted_run
    m = int(rp[-1] // 2)
    members, best = oracle.pareto_front(st, m)
    k1, k2 = st.k1[members], st.k2[members]
    for a in range(members.size):
        dom = (k1 <= k1[a]) & (k2 <= k2[a]) & ((k1 < k1[a]) | (k2 < k2[a]))
        assert not dom.any()
    q = [1.0 - oracle.objective_values(m, int(a), int(b))[0] - oracle.objective_values(m, int(a), int(b))[1]
         for a, b in zip(k1, k2)]
    assert q[best] == max(q)
    # Every other individual of P is dominated by a front member.
    others = np.setdiff1d(np.arange(st.k1.size), members)
    for p in others:
        dom = (k1 <= st.k1[p]) & (k2 <= st.k2[p]) & ((k1 < st.k1[p]) | (k2 < st.k2[p]))
        assert dom.any()


def test_keys_match_labels_and_progress(oracle, planted, planted_run):
    rp, ci, _ = planted
    _, st0, st = planted_run
    m = rp[-1] // 2
    intra, S = oracle.objectives(rp, ci, st.labels)
    assert np.array_equal(st.k1, m - intra) and np.array_equal(st.k2, S)
    q0 = (4 * m * st0.k1 + st0.k2).min()
    q1 = (4 * m * st.k1 + st.k2).min()
    assert q1 < q0


def test_reproducible_and_resumable(oracle):
    rp, ci, _ = synth.planted_partition(5, 30, 0.3, 0.02, seed=4)
    params = oracle.Params(pop_size=24, seed=77)
    st0 = oracle.population_init(rp, ci, params)
    a = oracle.run(rp, ci, params, st0, 6)
    b = oracle.run(rp, ci, params, oracle.run(rp, ci, params, st0, 2), 4)
    assert a.generation == b.generation == 6
    assert np.array_equal(a.labels, b.labels) and np.array_equal(a.k1, b.k1)
    c = oracle.run(rp, ci, oracle.Params(pop_size=24, seed=78), st0, 6)
    assert not np.array_equal(a.labels, c.labels)


def test_threaded_helpers_match_the_sequential_oracle(oracle):
    """The test-side helpers that split a generation's children (or a set of
    labellings) over host threads give exactly what the sequential oracle
    gives: same offspring, same keys, same next population."""
    import synth
    rp, ci = synth.lfr_style(2000, 12, 30, 0.3, seed=3)[:2]
    params = oracle.Params(pop_size=30, seed=77)
    st = oracle.population_init(rp, ci, params)
    seq = oracle.run(rp, ci, params, st, 3)
    par = oracle.run_parallel(rp, ci, params, st, 3, threads=5)
    assert par.generation == seq.generation == 3
    assert np.array_equal(par.labels, seq.labels)
    assert np.array_equal(par.k1, seq.k1) and np.array_equal(par.k2, seq.k2)
    Q, a, b = oracle.make_offspring(rp, ci, params, 4, seq)
    Q2, a2, b2 = oracle.make_offspring_parallel(rp, ci, params, 4, seq, threads=7)
    assert np.array_equal(Q, Q2) and np.array_equal(a, a2) and np.array_equal(b, b2)
    i1, s1 = oracle.objectives(rp, ci, Q)
    i2, s2 = oracle.objectives_parallel(rp, ci, Q, threads=3)
    assert np.array_equal(i1, i2) and np.array_equal(s1, s2)
