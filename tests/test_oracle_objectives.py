"""Pins for the oracle's objectives, Eq. (objectives) (not gpu)."""
from fractions import Fraction

import numpy as np
import pytest

import synth
from _golden import frac, graph, ints, load


def test_fig2_toy_graph(oracle):
    d = load("fig2_toy_graph.txt")
    rp, ci = graph(d)
    m = rp[-1] // 2
    assert m == int(d["m"])
    intra, S = oracle.objectives(rp, ci, ints(d["labels"]))
    assert intra[0] == int(d["intra"]) and S[0] == int(d["sumsq"])
    assert Fraction(int(m - intra[0]), int(m)) == frac(d["f1"])
    assert Fraction(int(S[0]), int(4 * m * m)) == frac(d["f2"])
    f1, f2 = oracle.objective_values(int(m), int(m - intra[0]), int(S[0]))
    assert f1 == float(frac(d["f1"])) and f2 == float(frac(d["f2"]))


def test_appendix_e_objectives(oracle):
    d = load("appE_operator_example.txt")
    rp, ci = graph(d)
    m = int(rp[-1] // 2)
    for tag in ("child", "mutated"):
        intra, S = oracle.objectives(rp, ci, ints(d[tag]))
        assert intra[0] == int(d[f"{tag}_intra"]) and S[0] == int(d[f"{tag}_sumsq"])
        assert Fraction(m - int(intra[0]), m) == frac(d[f"{tag}_f1"])
        assert Fraction(int(S[0]), 4 * m * m) == frac(d[f"{tag}_f2"])


@pytest.fixture(scope="module")
def small_graph():
    return synth.lfr_style(600, 12, 30, 0.3, cmin=10, cmax=60, seed=3)


def test_closed_forms(oracle, small_graph):
    rp, ci, _ = small_graph
    n = rp.size - 1
    m = int(rp[-1] // 2)
    deg = np.diff(rp)
    # One community: every edge internal, D = 2m -> (f1, f2) = (0, 1).
    intra, S = oracle.objectives(rp, ci, np.full(n, 5, np.int32))
    assert intra[0] == m and S[0] == 4 * m * m
    # Singletons: no internal edge, D_v = deg v -> (1, sum deg^2 / 4m^2).
    intra, S = oracle.objectives(rp, ci, np.arange(n, dtype=np.int32))
    assert intra[0] == 0 and S[0] == int((deg.astype(np.int64) ** 2).sum())


def test_modularity_identity_networkx(oracle, small_graph):
    """1 - f1 - f2 equals Newman modularity (Eq. modularity), via networkx."""
    nx = pytest.importorskip("networkx")
    rp, ci, truth = small_graph
    n = rp.size - 1
    m = int(rp[-1] // 2)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    src = np.repeat(np.arange(n), np.diff(rp))
    G.add_edges_from((int(a), int(b)) for a, b in zip(src, ci) if a < b)
    labs = [truth] + list(synth.random_labels(n, 3, seed=1, n_distinct=8)) + [synth.random_labels(n, 1, 2)[0]]
    for lab in labs:
        intra, S = oracle.objectives(rp, ci, lab)
        f1, f2 = oracle.objective_values(m, int(m - intra[0]), int(S[0]))
        comms = {}
        for v, c in enumerate(lab):
            comms.setdefault(int(c), set()).add(v)
        q = nx.algorithms.community.modularity(G, list(comms.values()))
        assert abs((1.0 - f1 - f2) - q) < 1e-12


def test_label_permutation_invariance(oracle, small_graph):
    rp, ci, _ = small_graph
    n = rp.size - 1
    rng = np.random.default_rng(4)
    lab = synth.random_labels(n, 1, 5, n_distinct=40)[0]
    perm = rng.permutation(n).astype(np.int32)
    a = oracle.objectives(rp, ci, lab)
    b = oracle.objectives(rp, ci, perm[lab])
    assert a[0][0] == b[0][0] and a[1][0] == b[1][0]


def test_degree_totals_and_bounds(oracle, small_graph):
    rp, ci, _ = small_graph
    n = rp.size - 1
    m = int(rp[-1] // 2)
    labs = synth.random_labels(n, 5, 9, n_distinct=20)
    intra, S = oracle.objectives(rp, ci, labs)
    deg = np.diff(rp)
    for r in range(5):
        D = np.bincount(labs[r], weights=deg, minlength=n)
        assert D.sum() == 2 * m
        assert 0 <= intra[r] <= m and 0 < S[r] <= 4 * m * m


def test_rejects_out_of_range_labels(oracle, small_graph):
    rp, ci, _ = small_graph
    n = rp.size - 1
    lab = np.zeros(n, np.int32)
    lab[7] = n
    with pytest.raises(RuntimeError):
        oracle.objectives(rp, ci, lab)
