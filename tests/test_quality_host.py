"""Pins for the quality helpers (NMI, AMI, pairwise F1) and the whole-run
quality smoke of the oracle on the planted workload (not gpu)."""
from itertools import combinations

import numpy as np
import pytest

import synth
from synth import quality


def _random_pairs():
    rng = np.random.default_rng(4)
    for n, ka, kb in [(10, 2, 3), (57, 5, 5), (300, 12, 7), (1000, 40, 60)]:
        yield rng.integers(0, ka, n), rng.integers(0, kb, n)
    truth = np.repeat(np.arange(10), 30)
    noisy = truth.copy()
    noisy[rng.choice(300, 40, replace=False)] = rng.integers(0, 10, 40)
    yield noisy, truth


def test_nmi_special_cases():
    a = np.array([0, 0, 1, 1, 2, 2])
    assert quality.nmi(a, a) == pytest.approx(1.0, abs=1e-15)
    assert quality.nmi(a, 7 - 3 * a) == pytest.approx(1.0, abs=1e-15)  # relabelled
    assert quality.nmi([0, 0, 1, 1], [0, 1, 0, 1]) == pytest.approx(0.0, abs=1e-15)  # independent
    assert quality.nmi(np.zeros(5), np.zeros(5)) == 1.0
    assert quality.nmi(np.zeros(4), [0, 0, 1, 1]) == 0.0


def test_nmi_two_by_two_by_hand():
    """M = [[2, 0], [1, 1]], N = 4: MI = 1/2 ln 4/3 + 1/4 ln 2/3 + 1/4 ln 2,
    H(a) = ln 2, H(b) = ln 4 - 3/4 ln 3."""
    mi = 0.5 * np.log(4 / 3) + 0.25 * np.log(2 / 3) + 0.25 * np.log(2)
    ha, hb = np.log(2), np.log(4) - 0.75 * np.log(3)
    assert quality.nmi([0, 0, 1, 1], [0, 0, 0, 1]) == pytest.approx(2 * mi / (ha + hb), rel=1e-14)


def test_nmi_ami_against_scikit_learn():
    metrics = pytest.importorskip("sklearn.metrics")
    for a, b in _random_pairs():
        assert quality.nmi(a, b) == pytest.approx(
            metrics.normalized_mutual_info_score(a, b, average_method="arithmetic"), abs=1e-12)
        assert quality.ami(a, b) == pytest.approx(
            metrics.adjusted_mutual_info_score(a, b, average_method="max"), abs=1e-9)


def test_ami_special_cases():
    a = np.repeat(np.arange(4), 5)
    assert quality.ami(a, a) == pytest.approx(1.0, abs=1e-12)
    assert quality.ami(np.zeros(6), np.zeros(6)) == 1.0
    # A random labeling scores near 0 on average (E[MI] is subtracted).
    rng = np.random.default_rng(0)
    vals = [quality.ami(a.repeat(10), rng.integers(0, 4, 200)) for _ in range(20)]
    assert abs(np.mean(vals)) < 0.01


def test_expected_mutual_information_brute_force():
    """E[MI] over every relabelling of a 6-node partition with sizes (3, 2, 1)
    against a fixed one with sizes (2, 2, 2): the hypergeometric formula equals
    the mean MI over all 6!/(3!2!1!) = 60 distinct assignments."""
    from itertools import permutations
    fixed = np.array([0, 0, 1, 1, 2, 2])
    seen = set(permutations([0, 0, 0, 1, 1, 2]))
    mis = [quality._mutual_information(quality.contingency(np.array(p), fixed)) for p in seen]
    M = quality.contingency(np.array([0, 0, 0, 1, 1, 2]), fixed)
    assert len(seen) == 60
    assert quality.expected_mutual_information(M) == pytest.approx(np.mean(mis), rel=1e-12)


def test_pairwise_f1_brute_force():
    for pred, truth in _random_pairs():
        if pred.size > 60:
            continue
        tp = pp = tt = 0
        for x, y in combinations(range(pred.size), 2):
            sp, st = pred[x] == pred[y], truth[x] == truth[y]
            tp += sp and st
            pp += sp
            tt += st
        p, r = tp / pp, tp / tt
        assert quality.pairwise_f1(pred, truth) == pytest.approx(2 * p * r / (p + r), rel=1e-14)
    assert quality.pairwise_f1(np.arange(5), np.arange(5)) == 1.0
    assert quality.pairwise_f1(np.arange(5), np.zeros(5)) == 0.0


@pytest.mark.parametrize("init_mode", [0, 1])
def test_oracle_recovers_planted_partition(oracle, init_mode):
    """The tiny workload (planted partition, 10 x 100 nodes, N_p = 100,
    G = 100): the recommended member of the final front recovers the planted
    communities (NMI >= 0.9; the paper reports NMI near 1 at low mixing)."""
    rp, ci, truth = synth.workload("planted-1k", seed=0)
    p = oracle.Params(seed=0, init_mode=init_mode)
    st = oracle.run(rp, ci, p, oracle.population_init(rp, ci, p), 100)
    members, best = oracle.pareto_front(st, int(rp[-1] // 2))
    labels = st.labels[members[best]]
    assert quality.nmi(labels, truth) >= 0.9
    assert quality.ami(labels, truth) >= 0.9
    assert quality.pairwise_f1(labels, truth) >= 0.9
