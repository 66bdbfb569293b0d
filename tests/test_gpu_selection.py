"""GPU parity of the front's community statistics and the selection criteria
(Alg. 3 and the Sec. 4.4 alternatives): the CUDA path through the C ABI
against the oracle run on the same seeded inputs, bit for bit (the
conductance doubles compared as bit patterns)."""
import numpy as np
import pytest

import oracle
import paper_2506_01752_gb300 as mocd
import synth
from _golden import graph, load

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mocd.build.build()
    mocd.load()
    oracle.build()


def _star_plus():
    rng = np.random.default_rng(0)
    n = 300 + 1 + 40 + 5
    u = [0] * 300 + list(rng.integers(1, n - 5, 600))
    v = list(range(1, 301)) + list(rng.integers(1, n - 5, 600))
    return synth.csr_from_edges(n, u, v)


GRAPHS = {
    "fig2": lambda: graph(load("fig2_toy_graph.txt")),
    "pair": lambda: synth.csr_from_edges(2, [0], [1]),
    "star": _star_plus,
    "planted-1k": lambda: synth.workload("planted-1k", seed=0)[:2],
    "lfr-3k": lambda: synth.lfr_style(3000, 20, 50, 0.3, seed=2)[:2],
    "lfr-40k": lambda: synth.workload("lfr-40k", seed=0, mu=0.5)[:2],
}


@pytest.mark.parametrize("gname,G,kw", [
    ("fig2", 0, dict(pop_size=13)),
    ("fig2", 5, dict(pop_size=64, n_parents=3)),
    ("pair", 3, dict(pop_size=9)),
    ("star", 4, dict(pop_size=24)),
    ("planted-1k", 0, dict(pop_size=100)),
    ("planted-1k", 30, dict(pop_size=100)),
    ("planted-1k", 5, dict(pop_size=128, init_mode=1)),
    ("lfr-3k", 20, dict(pop_size=100, seed=3)),
    ("lfr-40k", 3, dict(pop_size=100, seed=1)),
])
def test_front_stats_and_selection_match_oracle(gname, G, kw):
    rp, ci = GRAPHS[gname]()
    n, m = rp.size - 1, int(rp[-1] // 2)
    ref = oracle.population_init(rp, ci, oracle.Params(**kw))
    if G:
        ref = oracle.run(rp, ci, oracle.Params(**kw), ref, G)
    members, best = oracle.pareto_front(ref, m)
    ostats = oracle.community_stats(rp, ci, ref.labels[members])
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, mocd.Params(**kw))
        mocd.generation(h, G)
        st = mocd.front_stats(h)
        assert np.array_equal(st.communities, ostats[0])
        assert np.array_equal(st.size_sumsq, ostats[1])
        assert np.array_equal(st.mean_conductance.view(np.uint64), ostats[2].view(np.uint64))
        assert np.array_equal(st.max_conductance.view(np.uint64), ostats[3].view(np.uint64))
        k = ostats[0]
        targets = sorted({1, int(k.min()), int(np.median(k)), int(k.max()) + 5})
        for criterion in range(5):
            for target in (targets if criterion == mocd.SELECT_COMMUNITIES else [0]):
                want = oracle.select_solution(m, n, ref.k1[members], ref.k2[members], ostats, criterion, target)
                assert mocd.select_solution(h, criterion, target) == want, (criterion, target)
        assert mocd.select_solution(h, mocd.SELECT_MODULARITY) == mocd.pareto_front(h, False).best == best
    finally:
        mocd.destroy(h)


def test_selection_rejects_bad_arguments():
    rp, ci = GRAPHS["planted-1k"]()
    h = mocd.graph_upload(rp, ci)
    try:
        with pytest.raises(mocd.MocdError) as e:
            mocd.front_stats(h)
        assert e.value.status == -9  # no population yet
        mocd.population_init(h, mocd.Params(pop_size=8))
        for crit, target in ((5, 0), (-1, 0), (mocd.SELECT_COMMUNITIES, 0)):
            with pytest.raises(mocd.MocdError) as e:
                mocd.select_solution(h, crit, target)
            assert e.value.status == -1
    finally:
        mocd.destroy(h)


def test_stats_repeatable_with_reused_and_regrown_scratch():
    """Stats of the same front twice (scratch reused) and again after the
    population grew (scratch regrown) agree with a fresh context."""
    rp, ci = GRAPHS["lfr-3k"]()
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, mocd.Params(pop_size=16, seed=2))
        mocd.generation(h, 4)
        a = mocd.front_stats(h)
        b = mocd.front_stats(h)
        mocd.population_init(h, mocd.Params(pop_size=100, seed=2))
        mocd.generation(h, 4)
        c = mocd.front_stats(h)
    finally:
        mocd.destroy(h)
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, mocd.Params(pop_size=100, seed=2))
        mocd.generation(h, 4)
        d = mocd.front_stats(h)
    finally:
        mocd.destroy(h)
    for x, y in ((a, b), (c, d)):
        for f in ("communities", "size_sumsq", "mean_conductance", "max_conductance"):
            assert np.array_equal(getattr(x, f), getattr(y, f))
