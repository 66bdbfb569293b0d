"""Late-generation parity at full size (checkpoint-resume).

A whole oracle run of G = 100 generations at n = 10^6 would take hours on one
core, so the late generations are checked by resuming: the GPU runs G - 1
generations of Alg. 1, its population P^(G-1) is read back (labels and exact
keys, which are themselves checked against the oracle's objectives), the
oracle computes generation G from that state, and the GPU's generation G --
the offspring Q (child order, before selection), the next population and its
Pareto front -- must match bit for bit. This covers the mutation paths that
only a converged population exercises (the Misra-Gries shortcut that settles
most pairs, the recount, the hub count tables) at the configurations' own
sizes and launch shapes. One full G = 100 oracle run at n = 40,000 closes the
chain from generation 0.
"""
import functools
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import paper_2506_01752_gb300 as mocd
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mocd.build.build()
    mocd.load()
    oracle.build()


@functools.lru_cache(maxsize=None)
def _lfr_40k(mu):
    return synth.workload("lfr-40k", seed=1, mu=mu)[:2]


def _compare_front(h, ref, m):
    fr = mocd.pareto_front(h)
    members, best = oracle.pareto_front(ref, m)
    assert fr.best == best, "recommended member differs"
    assert np.array_equal(fr.labels, ref.labels[members]), "front labels differ"
    assert np.array_equal(fr.intra, m - ref.k1[members]) and np.array_equal(fr.sumsq, ref.k2[members])
    for a in range(members.size):
        f1, f2 = oracle.objective_values(m, int(ref.k1[members[a]]), int(ref.k2[members[a]]))
        assert fr.f1[a] == f1 and fr.f2[a] == f2


def _resume_check(h, rp, ci, op, G, threads=None):
    """The GPU context has run G - 1 generations: check generation G."""
    m = int(rp[-1] // 2)
    labels, k1, k2, gen = mocd.get_population(h)
    assert gen == G - 1
    intra, S = oracle.objectives_parallel(rp, ci, labels, threads)
    assert np.array_equal(k1, m - intra) and np.array_equal(k2, S), "keys of P^(G-1) differ from the objectives"
    st = oracle.State(labels, k1, k2, gen)
    del labels
    mocd.generation(h, 1)
    q, qk1, qk2 = mocd.get_offspring(h)
    Q, rk1, rk2 = oracle.make_offspring_parallel(rp, ci, op, G, st, threads)
    assert np.array_equal(qk1, rk1) and np.array_equal(qk2, rk2), "offspring keys differ"
    bad = np.flatnonzero((q != Q).any(axis=1))
    assert bad.size == 0, f"offspring labels differ for children {bad[:8].tolist()}"
    del q
    ref = oracle.next_state(st, Q, rk1, rk2)
    del Q, st
    labels, k1, k2, gen = mocd.get_population(h)
    assert gen == G
    assert np.array_equal(k1, ref.k1) and np.array_equal(k2, ref.k2), "P^(G) keys differ"
    assert np.array_equal(labels, ref.labels), "P^(G) labels differ"
    del labels
    _compare_front(h, ref, m)


@pytest.mark.parametrize("mu", [0.1, 0.3, 0.7])
def test_lfr_40k_generation_100(mu):
    """The plain-method workload (n = 40,000 LFR-style, N_p = 100) at the end
    of its G = 100 run, across the mixing range."""
    rp, ci = _lfr_40k(mu)
    gp, op = mocd.Params(seed=3), oracle.Params(seed=3)
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, gp)
        mocd.generation(h, 99)
        _resume_check(h, rp, ci, op, 100)
    finally:
        mocd.destroy(h)


def test_lfr_40k_full_run_from_generation_0():
    """One whole G = 100 oracle run from the initial population (mu = 0.3):
    the GPU's population and front after generation 100 are bit-exact."""
    rp, ci = _lfr_40k(0.3)
    m = int(rp[-1] // 2)
    gp, op = mocd.Params(seed=5), oracle.Params(seed=5)
    ref = oracle.run_parallel(rp, ci, op, oracle.population_init(rp, ci, op), 100)
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, gp)
        mocd.generation(h, 100)
        labels, k1, k2, gen = mocd.get_population(h)
        assert gen == 100
        assert np.array_equal(k1, ref.k1) and np.array_equal(k2, ref.k2)
        assert np.array_equal(labels, ref.labels)
        _compare_front(h, ref, m)
    finally:
        mocd.destroy(h)


def test_lfr_1m_generation_100():
    """The large plain run (n = 10^6, m ~ 7.9M, maximum degree 200) at
    generation 100, in the engine's own launch configuration."""
    rp, ci, _ = synth.workload("lfr-1m", seed=0)
    gp, op = mocd.Params(seed=0), oracle.Params(seed=0)
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, gp)
        mocd.generation(h, 99)
        _resume_check(h, rp, ci, op, 100)
    finally:
        mocd.destroy(h)


def test_batch64_every_job_generation_20():
    """The batched-jobs workload (64 uneven jobs, n 1e3-5e4, N_p = 100 each)
    in the autotuned launch shape with the multi-member launches (form 2):
    every one of the 64 jobs at generation 20 of a batched run, offspring,
    population and front bit for bit."""
    G = 20
    insts = synth.batch_instances(64, seed=0)
    ctxs = [mocd.graph_upload(rp, ci) for rp, ci, _, _ in insts]
    try:
        for k, c in enumerate(ctxs):
            mocd.population_init(c, mocd.Params(seed=k))
        b = mocd.batch_create(ctxs)
        mocd.batch_autotune(b, 1)
        shape, _ = mocd.batch_form(b)
        mocd.batch_destroy(b)
        for k, c in enumerate(ctxs):
            mocd.population_init(c, mocd.Params(seed=k))
        b = mocd.batch_create(ctxs)
        try:
            mocd.batch_configure(b, shape, 2)
            mocd.batch_generation(b, G - 1)
            mocd.batch_synchronize(b)
            states = []
            for c in ctxs:
                labels, k1, k2, gen = mocd.get_population(c)
                assert gen == G - 1
                states.append(oracle.State(labels, k1, k2, gen))
            mocd.batch_generation(b, 1)
            mocd.batch_synchronize(b)
        finally:
            mocd.batch_destroy(b)

        def ref_of(k):
            rp, ci, _, _ = insts[k]
            op = oracle.Params(seed=k)
            st = states[k]
            m = int(rp[-1] // 2)
            intra, S = oracle.objectives(rp, ci, st.labels)
            assert np.array_equal(st.k1, m - intra) and np.array_equal(st.k2, S), k
            Q, rk1, rk2 = oracle.make_offspring(rp, ci, op, G, st)
            return Q, rk1, rk2, oracle.next_state(st, Q, rk1, rk2)

        with ThreadPoolExecutor(16) as ex:
            refs = list(ex.map(ref_of, range(len(insts))))
        for k, (c, (Q, rk1, rk2, ref)) in enumerate(zip(ctxs, refs)):
            rp = insts[k][0]
            q, qk1, qk2 = mocd.get_offspring(c)
            assert np.array_equal(qk1, rk1) and np.array_equal(qk2, rk2), k
            assert np.array_equal(q, Q), k
            labels, k1, k2, gen = mocd.get_population(c)
            assert gen == G
            assert np.array_equal(k1, ref.k1) and np.array_equal(k2, ref.k2), k
            assert np.array_equal(labels, ref.labels), k
            _compare_front(c, ref, int(rp[-1] // 2))
    finally:
        for c in ctxs:
            mocd.destroy(c)


def test_server_mix_with_a_large_job():
    """The serving workload's shape: a continuous-batching server running a
    job on an n = 120,000 LFR-style graph (average degree 16, maximum 200,
    communities 20-2000) for G = 100 together with smaller jobs. Each job's
    front equals the same job run alone; the large job run alone is checked
    against the oracle at generation 100 (resume), the small ones by whole
    oracle runs."""
    big = synth.lfr_style(120_000, 16, 200, 0.35, cmin=20, cmax=2000, seed=11)[:2]
    small = [
        (synth.lfr_style(2000, 16, 50, 0.2, seed=12)[:2], dict(seed=21), 100),
        (synth.workload("planted-1k", seed=0)[:2], dict(seed=22), 100),
        (synth.lfr_style(5000, 16, 50, 0.5, seed=13)[:2], dict(seed=23, pop_size=64), 60),
    ]
    jobs = [(big, dict(seed=20), 100)] + small
    srv = mocd.Server(1 << 34, max_running=3, depth=4)
    srv.start(admission_threads=2, policy=0)
    try:
        ids = [srv.submit(rp, ci, mocd.Params(**kw), G) for (rp, ci), kw, G in jobs]
        t_end = time.time() + 300
        while not all(srv.state(j)[0] >= mocd.Server.DONE for j in ids):
            assert time.time() < t_end, "server did not finish"
            srv.step()
            time.sleep(0.001)
        results = [srv.result(j) for j in ids]
        assert all(srv.state(j) == (mocd.Server.DONE, 0) for j in ids)
    finally:
        srv.close()
    # the large job alone, checked against the oracle at generation 100
    (rp, ci), kw, G = jobs[0]
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, mocd.Params(**kw))
        mocd.generation(h, G - 1)
        _resume_check(h, rp, ci, oracle.Params(**kw), G)
        alone = mocd.pareto_front(h)
    finally:
        mocd.destroy(h)
    got = results[0]
    assert got.best == alone.best and np.array_equal(got.labels, alone.labels)
    assert np.array_equal(got.intra, alone.intra) and np.array_equal(got.sumsq, alone.sumsq)
    assert np.array_equal(got.f1, alone.f1) and np.array_equal(got.f2, alone.f2)
    for ((rp, ci), kw, G), got in zip(small, results[1:]):
        op = oracle.Params(**kw)
        st = oracle.run_parallel(rp, ci, op, oracle.population_init(rp, ci, op), G)
        members, best = oracle.pareto_front(st, int(rp[-1] // 2))
        assert got.best == best and np.array_equal(got.labels, st.labels[members])
        assert np.array_equal(got.intra, int(rp[-1] // 2) - st.k1[members])
