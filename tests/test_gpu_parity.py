"""GPU parity: the CUDA path, called through the C ABI, against the CPU
oracle on the same seeded inputs. Everything here is integer or a single IEEE
division per value, so the bar is bit-exact equality: labels, integer keys
(m - intra, S), f1/f2 doubles, front membership and the recommended member.
"""
import numpy as np
import pytest

import oracle
import paper_2506_01752_gb300 as mocd
import synth
from _golden import graph, ints, load

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mocd.build.build()
    mocd.load()
    oracle.build()


class Ctx:
    def __init__(self, rp, ci):
        self.rp, self.ci = rp, ci
        self.h = mocd.graph_upload(rp, ci)

    def __enter__(self):
        return self.h

    def __exit__(self, *a):
        mocd.destroy(self.h)


def star_plus(n_leaves=300, extra=40, seed=0):
    """A hub of degree n_leaves (> 32, the count-table path) plus a random
    sparse part and isolated nodes (degree 0)."""
    rng = np.random.default_rng(seed)
    n = n_leaves + 1 + extra + 5
    u = [0] * n_leaves
    v = list(range(1, n_leaves + 1))
    a = rng.integers(1, n - 5, 600)
    b = rng.integers(1, n - 5, 600)
    rp, ci = synth.csr_from_edges(n, np.concatenate([u, a]), np.concatenate([v, b]))
    return rp, ci


def hub_of_degree(d, extra=300, seed=0):
    """Node 0 adjacent to nodes 1..d, plus a sparse random part among them."""
    rng = np.random.default_rng(seed)
    n = d + 1
    a = rng.integers(1, n, extra)
    b = rng.integers(1, n, extra)
    return synth.csr_from_edges(n, np.concatenate([np.zeros(d, np.int64), a]),
                                np.concatenate([np.arange(1, n), b]))


def degree_ladder(degrees=(1, 2, 7, 8, 9, 15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129)):
    """Disjoint stars whose centres have the given degrees: the boundaries of
    the mutation vote's per-lane sorting networks (8, 16, 32 entries), of the
    warp sort (33..64) and of the count table (65 and up). With random labels
    every neighbour label of a centre is distinct, so its votes tie widely
    (deep tie ranks)."""
    u, v, base = [], [], 0
    for d in degrees:
        u += [base] * d
        v += list(range(base + 1, base + 1 + d))
        base += d + 1
    return synth.csr_from_edges(base, u, v)


def complete_graph(k):
    u, v = np.triu_indices(k, 1)
    return synth.csr_from_edges(k, u, v)


GRAPHS = {
    "fig2": lambda: graph(load("fig2_toy_graph.txt")),
    "appE": lambda: graph(load("appE_operator_example.txt")),
    "planted-1k": lambda: synth.workload("planted-1k", seed=0)[:2],
    "lfr-3k": lambda: synth.lfr_style(3000, 20, 50, 0.3, seed=2)[:2],
    "star": lambda: star_plus(),
    "pair": lambda: synth.csr_from_edges(2, [0], [1]),
    # every degree in 33..64 (the sorting-network vote of the mutation
    # fallback), 65..128 and 129..256 (its shared count table)
    "dense": lambda: synth.planted_partition(2, 80, 0.5, 0.1, seed=5)[:2],
    "dense128": lambda: synth.planted_partition(2, 150, 0.6, 0.1, seed=7)[:2],
    "dense256": lambda: synth.planted_partition(2, 260, 0.65, 0.12, seed=8)[:2],
}


@pytest.mark.parametrize("gname", list(GRAPHS))
@pytest.mark.parametrize("kind", ["uniform", "few", "one", "singletons"])
def test_evaluate_matches_oracle(gname, kind):
    rp, ci = GRAPHS[gname]()
    n = rp.size - 1
    if kind == "uniform":
        lab = synth.random_labels(n, 7, seed=3)
    elif kind == "few":
        lab = synth.random_labels(n, 5, seed=4, n_distinct=min(n, 6))
    elif kind == "one":
        lab = np.full((1, n), n - 1, np.int32)
    else:
        lab = np.arange(n, dtype=np.int32)[None, :]
    with Ctx(rp, ci) as h:
        gi, gs = mocd.evaluate(h, lab)
    oi, os_ = oracle.objectives(rp, ci, lab)
    assert np.array_equal(gi, oi) and np.array_equal(gs, os_)


def test_evaluate_large_batches_and_lfr_40k():
    rp, ci, _ = synth.workload("lfr-40k", seed=0)
    n = rp.size - 1
    lab = np.concatenate([synth.random_labels(n, 70, seed=5),
                          synth.random_labels(n, 70, seed=6, n_distinct=900)])  # 140 > one batch of 128
    with Ctx(rp, ci) as h:
        gi, gs = mocd.evaluate(h, lab)
    oi, os_ = oracle.objectives(rp, ci, lab)
    assert np.array_equal(gi, oi) and np.array_equal(gs, os_)


def test_evaluate_rejects_out_of_range():
    rp, ci = GRAPHS["planted-1k"]()
    n = rp.size - 1
    lab = np.zeros((2, n), np.int32)
    lab[1, 5] = n
    with Ctx(rp, ci) as h:
        with pytest.raises(mocd.MocdError) as e:
            mocd.evaluate(h, lab)
        assert e.value.status == -1


def _params(**kw):
    return mocd.Params(**kw), oracle.Params(**kw)


def _compare_state(h, ref, m):
    labels, k1, k2, gen = mocd.get_population(h)
    assert gen == ref.generation
    assert np.array_equal(k1, ref.k1), "k1 differs"
    assert np.array_equal(k2, ref.k2), "k2 differs"
    assert np.array_equal(labels, ref.labels), "labels differ"
    fr = mocd.pareto_front(h)
    members, best = oracle.pareto_front(ref, m)
    assert fr.best == best
    assert np.array_equal(fr.labels, ref.labels[members])
    assert np.array_equal(fr.intra, m - ref.k1[members]) and np.array_equal(fr.sumsq, ref.k2[members])
    for a in range(members.size):
        f1, f2 = oracle.objective_values(m, int(ref.k1[members[a]]), int(ref.k2[members[a]]))
        assert fr.f1[a] == f1 and fr.f2[a] == f2


@pytest.mark.parametrize("init_mode", [0, 1])
@pytest.mark.parametrize("gname", ["fig2", "appE", "pair", "star", "planted-1k", "lfr-3k"])
def test_init_matches_oracle(gname, init_mode):
    rp, ci = GRAPHS[gname]()
    gp, op = _params(pop_size=37, seed=11, init_mode=init_mode)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, gp)
        _compare_state(h, oracle.population_init(rp, ci, op), int(rp[-1] // 2))


@pytest.mark.parametrize("gname,G,kw", [
    ("appE", 6, dict(pop_size=8)),
    ("fig2", 6, dict(pop_size=13, n_parents=3)),
    ("pair", 4, dict(pop_size=5)),
    ("star", 4, dict(pop_size=24)),
    ("star", 3, dict(pop_size=16, p_mutation=1.0)),
    ("planted-1k", 5, dict(pop_size=100)),
    ("planted-1k", 3, dict(pop_size=128, n_parents=16)),
    ("planted-1k", 3, dict(pop_size=1)),
    ("planted-1k", 3, dict(pop_size=2, n_parents=1)),
    ("planted-1k", 3, dict(pop_size=33, n_parents=5, p_crossover=1.0, p_mutation=0.0)),
    ("planted-1k", 3, dict(pop_size=31, n_parents=8, p_crossover=0.0, p_mutation=1.0)),
    ("lfr-3k", 4, dict(pop_size=100, seed=5)),
    # tiny graphs with large populations: many identical keys, multi-member fronts
    ("appE", 4, dict(pop_size=128)),
    ("pair", 3, dict(pop_size=100)),
    ("fig2", 5, dict(pop_size=127, n_parents=2)),
    ("fig2", 4, dict(pop_size=64, n_parents=7, p_mutation=0.5)),
    ("dense", 5, dict(pop_size=100)),
    ("dense", 3, dict(pop_size=64, p_mutation=1.0, seed=3)),
    ("dense128", 4, dict(pop_size=100)),
    ("dense128", 2, dict(pop_size=48, p_mutation=1.0, seed=4)),
    ("dense256", 3, dict(pop_size=64)),
    ("dense256", 2, dict(pop_size=32, p_mutation=1.0, seed=5)),
    # hybrid initialisation (singletons + one neighbour-majority step)
    ("star", 3, dict(pop_size=24, init_mode=1)),
    ("planted-1k", 4, dict(pop_size=100, init_mode=1)),
    ("lfr-3k", 3, dict(pop_size=64, n_parents=4, seed=7, init_mode=1)),
])
def test_generations_match_oracle(gname, G, kw):
    rp, ci = GRAPHS[gname]()
    gp, op = _params(**kw)
    m = int(rp[-1] // 2)
    ref = oracle.population_init(rp, ci, op)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, gp)
        for step in range(G):
            mocd.generation(h, 1)
            ref = oracle.run(rp, ci, op, ref, 1)
            _compare_state(h, ref, m)


@pytest.mark.parametrize("gname,G,kw", [
    ("hub512", 3, dict(pop_size=24, p_mutation=1.0)),       # the largest degree of the shared count table
    ("hub512", 2, dict(pop_size=40, seed=(1 << 40) + 7)),
    ("one-edge", 3, dict(pop_size=20, p_mutation=1.0)),     # thousands of isolated nodes
    ("k40", 4, dict(pop_size=30, p_mutation=0.5)),          # one dense community, degree 39
    ("k33", 3, dict(pop_size=16, p_mutation=1.0)),          # degree exactly 32
    ("ladder", 3, dict(pop_size=40, p_mutation=1.0)),      # network-size boundaries, two rounds of pairs
    ("ladder", 4, dict(pop_size=100, seed=9)),
    ("lfr-3k", 2, dict(pop_size=50, seed=0xDEADBEEF12345678)),  # both key words non-zero
    # the degree 33..64 vote sorts as many entries as the graph's largest
    # degree needs (40, 48, 56 or 64): each size at both ends of its range
    ("ladder40", 3, dict(pop_size=40, p_mutation=1.0)),
    ("ladder48", 3, dict(pop_size=40, p_mutation=1.0)),
    ("ladder56", 3, dict(pop_size=40, p_mutation=1.0)),
    ("ladder64", 3, dict(pop_size=40, p_mutation=1.0)),
    ("k49", 3, dict(pop_size=30, p_mutation=0.5)),
    ("k57", 3, dict(pop_size=30, p_mutation=0.5)),
])
def test_extreme_graphs_match_oracle(gname, G, kw):
    rp, ci = {
        "hub512": lambda: hub_of_degree(512),
        "one-edge": lambda: synth.csr_from_edges(3000, [17], [2950]),
        "k40": lambda: complete_graph(40),
        "k33": lambda: complete_graph(33),
        "k49": lambda: complete_graph(49),
        "k57": lambda: complete_graph(57),
        "ladder": degree_ladder,
        "ladder40": lambda: degree_ladder((5, 33, 40)),
        "ladder48": lambda: degree_ladder((33, 41, 48)),
        "ladder56": lambda: degree_ladder((33, 49, 56)),
        "ladder64": lambda: degree_ladder((33, 57, 64)),
        "lfr-3k": GRAPHS["lfr-3k"],
    }[gname]()
    gp, op = _params(**kw)
    m = int(rp[-1] // 2)
    ref = oracle.population_init(rp, ci, op)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, gp)
        _compare_state(h, ref, m)
        for step in range(G):
            mocd.generation(h, 1)
            ref = oracle.run(rp, ci, op, ref, 1)
            _compare_state(h, ref, m)


def test_upload_rejects_asymmetric_graphs():
    """Symmetry is checked on the device after the per-row host checks: a
    missing mirror anywhere gives NOT_SYMMETRIC, a self loop elsewhere still
    gives SELF_LOOP (the host checks come first)."""
    cases = [(np.array([0, 1, 1]), np.array([1]))]  # 0 -> 1 without 1 -> 0
    rp, ci, _ = synth.lfr_style(20000, 20, 50, 0.3, seed=4)
    for row in (10, rp.size - 50):
        bad = ci.copy()
        nb = bad[rp[row]:rp[row + 1]]
        w = int(np.setdiff1d(np.arange(rp.size - 1), np.concatenate([nb, [row]]))[0])
        bad[rp[row]] = w  # row -> w without w -> row
        cases.append((rp, bad))
    for rp_, ci_ in cases:
        with pytest.raises(mocd.MocdError) as e:
            mocd.graph_upload(rp_, ci_)
        assert e.value.status == -2
    bad = cases[1][1].copy()
    last = rp.size - 10
    bad[rp[last]] = last  # and a self loop in a later row: the host check decides
    with pytest.raises(mocd.MocdError) as e:
        mocd.graph_upload(rp, bad)
    assert e.value.status == -3


@pytest.mark.parametrize("gname,G,kw", [
    ("hub2000", 3, dict(pop_size=24, p_mutation=1.0)),      # global count tables, every pair
    ("hub2000", 3, dict(pop_size=64, seed=3)),
    ("hub10000", 2, dict(pop_size=16, p_mutation=1.0)),
    ("hub-ladder", 3, dict(pop_size=40, p_mutation=1.0)),   # 511, 512 (shared table), 513, 1024 (global)
    ("lfr-hubs", 3, dict(pop_size=64, seed=2)),              # n = 100k, 263 nodes above 512, max 1709
])
def test_hub_degrees_match_oracle(gname, G, kw):
    """Degrees above the shared count table (512): the open votes of these
    hubs run in the hub kernel with count tables in global scratch; the
    paper's mutation has no degree limit (Sec. 4.3.2). Whole generations
    bit-exact against the oracle, and evaluation too."""
    rp, ci = {
        "hub2000": lambda: hub_of_degree(2000, extra=3000, seed=1),
        "hub10000": lambda: hub_of_degree(10000, extra=12000, seed=2),
        "hub-ladder": lambda: degree_ladder((1, 40, 100, 511, 512, 513, 1024)),
        "lfr-hubs": lambda: synth.lfr_style(100_000, 20, 2000, 0.3, cmin=20, cmax=3000, seed=3)[:2],
    }[gname]()
    gp, op = _params(**kw)
    m = int(rp[-1] // 2)
    ref = oracle.population_init(rp, ci, op)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, gp)
        _compare_state(h, ref, m)
        for step in range(G):
            mocd.generation(h, 1)
            ref = oracle.run_parallel(rp, ci, op, ref, 1)
            _compare_state(h, ref, m)
        lab = synth.random_labels(rp.size - 1, 3, seed=1)
        gi, gs = mocd.evaluate(h, lab)
        oi, os_ = oracle.objectives(rp, ci, lab)
        assert np.array_equal(gi, oi) and np.array_equal(gs, os_)


def test_planted_full_run_front_bit_exact():
    """The tiny workload: planted partition n = 1000, N_p = 100, G = 100."""
    rp, ci, truth = synth.workload("planted-1k", seed=0)
    gp, op = _params(seed=0)
    m = int(rp[-1] // 2)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, gp)
        mocd.generation(h, 100)
        ref = oracle.run(rp, ci, op, oracle.population_init(rp, ci, op), 100)
        _compare_state(h, ref, m)


@pytest.mark.parametrize("mu", [0.1, 0.4, 0.7])
def test_lfr_40k_generations_bit_exact(mu):
    """The benchmark graph shape (n = 40k, LFR-style) for a few generations."""
    rp, ci, _ = synth.workload("lfr-40k", seed=1, mu=mu)
    gp, op = _params(seed=3)
    m = int(rp[-1] // 2)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, gp)
        mocd.generation(h, 2)
        ref = oracle.run(rp, ci, op, oracle.population_init(rp, ci, op), 2)
        _compare_state(h, ref, m)


def test_resume_from_checkpoint_matches_uninterrupted():
    rp, ci = GRAPHS["lfr-3k"]()
    gp, op = _params(pop_size=40, seed=21)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, gp)
        mocd.generation(h, 3)
        labels, k1, k2, gen = mocd.get_population(h)
        mocd.generation(h, 3)
        full = mocd.get_population(h)
    with Ctx(rp, ci) as h2:
        mocd.set_population(h2, gp, labels, gen)
        assert np.array_equal(mocd.get_population(h2)[1], k1)
        mocd.generation(h2, 3)
        resumed = mocd.get_population(h2)
    assert resumed[3] == full[3] == 6
    for a, b in zip(resumed[:3], full[:3]):
        assert np.array_equal(a, b)
    # and the oracle agrees with the resumed state
    ref = oracle.run(rp, ci, op, oracle.State(labels, k1, k2, gen), 3)
    assert np.array_equal(resumed[0], ref.labels)


def test_appendix_e_state_one_generation():
    """Start from the App. E parents and check one generation against the oracle."""
    d = load("appE_operator_example.txt")
    rp, ci = graph(d)
    P = np.stack([ints(d["parent1"]), ints(d["parent2"]), ints(d["parent3"])] * 2)
    gp, op = _params(pop_size=6, n_parents=3, seed=2)
    m = int(rp[-1] // 2)
    with Ctx(rp, ci) as h:
        mocd.set_population(h, gp, P, 0)
        i, s = oracle.objectives(rp, ci, P)
        ref = oracle.State(P.copy(), m - i, s, 0)
        for _ in range(3):
            mocd.generation(h, 1)
            ref = oracle.run(rp, ci, op, ref, 1)
            _compare_state(h, ref, m)


def test_kernel_timing_reports_every_stage():
    rp, ci = GRAPHS["planted-1k"]()
    with Ctx(rp, ci) as h:
        mocd.population_init(h, mocd.Params())
        mocd.set_timing(h, True)
        mocd.generation(h, 2)
        t = mocd.kernel_times(h)
        assert set(t) == set(mocd.STAGES) and all(v >= 0 for v in t.values())
        # timing on or off does not change results
        a = mocd.get_population(h)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, mocd.Params())
        mocd.generation(h, 2)
        b = mocd.get_population(h)
    assert np.array_equal(a[0], b[0])


@pytest.mark.parametrize("degrees,expect", [
    ((5, 20, 32), 4),          # crossover, mutation, evaluation, selection
    ((5, 40), 5),              # + the degree 33..64 vote kernel
    ((100,), 5),               # + the degree 65..128 vote kernel
    ((300,), 4),               # 129..512: the mutation kernel's shared table
    ((600,), 5),               # + the hub kernel above 512
    ((40, 100, 300, 600), 7),  # every class at once
])
def test_generation_kernel_count(degrees, expect):
    rp, ci = degree_ladder(degrees)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, mocd.Params())
        mocd.set_timing(h, True)
        assert mocd.generation_kernels(h) == expect
        # counting captures the plain graph only; the timing graph still runs
        mocd.generation(h, 1)
        assert set(mocd.kernel_times(h)) == set(mocd.STAGES)


def test_timing_toggled_every_generation_matches_oracle():
    """The plain and the stage-timed generation graphs coexist; switching
    between them every generation (as the benchmark does) changes nothing in
    the results, and stage times exist only after a timed launch."""
    rp, ci = GRAPHS["lfr-3k"]()
    gp, op = _params(pop_size=40, seed=17)
    m = int(rp[-1] // 2)
    ref = oracle.population_init(rp, ci, op)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, gp)
        for step in range(6):
            timed = step % 2 == 1
            mocd.set_timing(h, timed)
            mocd.generation(h, 1)
            if timed:
                assert set(mocd.kernel_times(h)) == set(mocd.STAGES)
            else:
                with pytest.raises(mocd.MocdError) as e:
                    mocd.kernel_times(h)
                assert e.value.status == -9
            ref = oracle.run(rp, ci, op, ref, 1)
            _compare_state(h, ref, m)


def test_invalid_params_rejected():
    rp, ci = GRAPHS["planted-1k"]()
    with Ctx(rp, ci) as h:
        for bad in (dict(pop_size=0), dict(pop_size=129), dict(n_parents=17), dict(p_crossover=1.5),
                    dict(p_mutation=-0.1), dict(init_mode=3)):
            with pytest.raises(mocd.MocdError) as e:
                mocd.population_init(h, mocd.Params(**bad))
            assert e.value.status == -1
        with pytest.raises(mocd.MocdError) as e:
            mocd.generation(h, 1)
        assert e.value.status == -9


def test_offspring_match_oracle():
    """Q of generations 1 and 2 (child order, before selection) and their keys."""
    rp, ci = GRAPHS["lfr-3k"]()
    gp, op = _params(pop_size=64, seed=8)
    st = oracle.population_init(rp, ci, op)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, gp)
        with pytest.raises(mocd.MocdError):
            mocd.get_offspring(h)  # no generation yet
        for gen in (1, 2):
            mocd.generation(h, 1)
            q, qk1, qk2 = mocd.get_offspring(h)
            Q, rk1, rk2 = oracle.make_offspring(rp, ci, op, gen, st)
            assert np.array_equal(q, Q) and np.array_equal(qk1, rk1) and np.array_equal(qk2, rk2)
            st = oracle.run(rp, ci, op, st, 1)


def test_full_size_1m_sampled():
    """The large workload (n = 10^6, m ~ 7.9M, maximum degree 200) in the
    engine's own launch configuration: the whole initial population and its
    keys, then sampled children of generation 1, bit for bit."""
    rp, ci, _ = synth.workload("lfr-1m", seed=0)
    gp, op = _params(seed=0)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, gp)
        p0, k1, k2, _ = mocd.get_population(h)
        mocd.generation(h, 1)
        q, qk1, qk2 = mocd.get_offspring(h)
    st = oracle.population_init(rp, ci, op)
    assert np.array_equal(k1, st.k1) and np.array_equal(k2, st.k2)
    assert np.array_equal(p0, st.labels)
    del p0
    for i in (0, 57, 99):
        Q, rk1, rk2 = oracle.make_offspring_range(rp, ci, op, 1, st, i, i + 1)
        assert np.array_equal(q[i], Q[i]), f"child {i} differs"
        assert qk1[i] == rk1[i] and qk2[i] == rk2[i]


@pytest.mark.parametrize("n,kw,G", [
    (200_000, dict(pop_size=100, seed=2), 2),
    (170_000, dict(pop_size=128, n_parents=5, seed=3), 1),     # the widest population
    (400_000, dict(pop_size=50, seed=4, init_mode=1), 1),      # W = 52: a partial last int4
])
def test_label_matrix_beyond_l2_matches_oracle(n, kw, G):
    """Label matrices and degree histograms larger than half the L2 (so the
    histogram additions of the first generations miss it): initial
    population and whole generations bit-exact against the oracle, with
    populations of 100, 128 and 50 (a partial last int4 of labels)."""
    rp, ci, _ = synth.lfr_style(n, 16, 120, 0.3, cmin=20, cmax=1000, seed=n)
    assert ((kw["pop_size"] + 3) // 4 * 4) * n * 4 > 64 << 20
    gp, op = _params(**kw)
    m = int(rp[-1] // 2)
    ref = oracle.population_init(rp, ci, op)
    with Ctx(rp, ci) as h:
        mocd.population_init(h, gp)
        _compare_state(h, ref, m)
        mocd.generation(h, G)
        ref = oracle.run_parallel(rp, ci, op, ref, G)
        _compare_state(h, ref, m)
