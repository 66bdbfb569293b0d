"""Continuous-batching server: each job's front equals the same job run alone
(and the oracle's), whatever else is running, under a tight device-memory
budget too."""
import numpy as np
import pytest

import oracle
import paper_2506_01752_gb300 as mocd
import synth
from _golden import graph, load

pytestmark = pytest.mark.gpu


def _jobs():
    return [
        (synth.workload("planted-1k", seed=0)[:2], dict(pop_size=100, seed=1), 12),
        (synth.lfr_style(3000, 20, 50, 0.3, seed=2)[:2], dict(pop_size=64, seed=2), 8),
        (graph(load("appE_operator_example.txt")), dict(pop_size=8, n_parents=3, seed=3), 6),
        (synth.lfr_style(1500, 12, 60, 0.4, seed=4)[:2], dict(pop_size=100, seed=4), 10),
        (graph(load("fig2_toy_graph.txt")), dict(pop_size=33, seed=5), 0),
        (synth.planted_partition(6, 40, 0.3, 0.02, seed=6)[:2], dict(pop_size=50, seed=6), 15),
    ]


def _alone(rp, ci, kw, G):
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, mocd.Params(**kw))
        mocd.generation(h, G)
        return mocd.pareto_front(h)
    finally:
        mocd.destroy(h)


def _drain(srv, ids, max_running):
    import time
    t_end = time.time() + 120
    while time.time() < t_end:
        running, queued, done = srv.step()
        assert running <= max_running
        if all(srv.state(j)[0] >= mocd.Server.DONE for j in ids):
            return
        time.sleep(0.0005)
    raise AssertionError("server did not finish")


TIGHT = "tight"  # a budget just above the largest job's footprint: about one job at a time


@pytest.mark.parametrize("budget,max_running,background", [
    (1 << 34, 8, None), (TIGHT, 8, None), (1 << 34, 1, None),
    (1 << 34, 8, 0), (TIGHT, 4, 1)])
def test_server_results_equal_alone(budget, max_running, background):
    jobs = _jobs()
    if budget == TIGHT:
        budget = max(mocd.job_footprint(rp, kw.get("pop_size", 100)) for (rp, _), kw, _ in jobs) + (1 << 20)
    srv = mocd.Server(budget, max_running=max_running, depth=3)
    if background is not None:
        srv.start(admission_threads=2, policy=background)
    try:
        ids = [srv.submit(rp, ci, mocd.Params(**kw), G) for (rp, ci), kw, G in jobs]
        if background is None:
            assert srv.state(ids[0])[0] == mocd.Server.QUEUED
        _drain(srv, ids, max_running)
        for jid, ((rp, ci), kw, G) in zip(ids, jobs):
            assert srv.state(jid) == (mocd.Server.DONE, 0)
            got = srv.result(jid)
            ref = _alone(rp, ci, kw, G)
            assert got.best == ref.best
            assert np.array_equal(got.labels, ref.labels)
            assert np.array_equal(got.intra, ref.intra) and np.array_equal(got.sumsq, ref.sumsq)
            assert np.array_equal(got.f1, ref.f1) and np.array_equal(got.f2, ref.f2)
        if background is None:
            assert srv.state(ids[0])[0] == mocd.Server.DONE
        # and the oracle agrees with every one of them
        for jid, ((rp, ci), kw, G) in zip(ids, jobs):
            op = oracle.Params(**kw)
            st = oracle.run(rp, ci, op, oracle.population_init(rp, ci, op), G)
            members, best = oracle.pareto_front(st, int(rp[-1] // 2))
            got = srv.result(jid)
            assert got.best == best and np.array_equal(got.labels, st.labels[members])
    finally:
        srv.close()


def test_server_failures():
    srv = mocd.Server(2 << 20, max_running=4, depth=2)  # 2 MiB: the small jobs fit, planted-1k does not
    try:
        big_rp, big_ci, _ = synth.workload("planted-1k", seed=0)
        j_big = srv.submit(big_rp, big_ci, mocd.Params(), 5)          # footprint > budget
        j_bad = srv.submit([0, 1, 2], [0, 1], mocd.Params(pop_size=4), 5)  # self loops
        j_asym = srv.submit([0, 1, 1], [1], mocd.Params(pop_size=4), 5)  # 0 -> 1 only
        rp, ci = graph(load("appE_operator_example.txt"))
        j_ok = srv.submit(rp, ci, mocd.Params(pop_size=8), 5)
        _drain(srv, [j_big, j_bad, j_asym, j_ok], 4)
        assert srv.state(j_big) == (mocd.Server.FAILED, -6)
        assert srv.state(j_bad) == (mocd.Server.FAILED, -3)
        assert srv.state(j_asym) == (mocd.Server.FAILED, -2)
        assert srv.state(j_ok)[0] == mocd.Server.DONE
        with pytest.raises(mocd.MocdError) as e:
            srv.result(j_big)
        assert e.value.status == -6
    finally:
        srv.close()


@pytest.mark.parametrize("background", [False, True])
def test_server_cancel_queued_and_running(background):
    """A queued job cancelled at once; a running job cancelled between rounds
    gets no further generations and is retired with its device memory
    returned to the pool; the other jobs' results equal the same jobs alone."""
    import time
    jobs = _jobs()
    base, _ = mocd.debug_pool_usage()
    srv = mocd.Server(1 << 34, max_running=1, depth=2)
    if background:
        srv.start(admission_threads=1, policy=0)
    try:
        big = synth.lfr_style(20000, 16, 50, 0.3, seed=9)[:2]
        j_run = srv.submit(big[0], big[1], mocd.Params(seed=1), 5000)   # long enough to be running
        ids = [srv.submit(rp, ci, mocd.Params(**kw), G) for (rp, ci), kw, G in jobs]
        j_queued = ids[1]
        srv.cancel(j_queued)
        assert srv.state(j_queued) == (mocd.Server.CANCELLED, -11)
        t_end = time.time() + 60
        while srv.state(j_run)[0] != mocd.Server.RUNNING:
            assert time.time() < t_end
            srv.step()
            time.sleep(0.001)
        for _ in range(5):
            srv.step()
        srv.cancel(j_run)
        srv.cancel(j_run)  # cancelling again is harmless
        _drain(srv, [j_run] + ids, 1)
        assert srv.state(j_run) == (mocd.Server.CANCELLED, -11)
        with pytest.raises(mocd.MocdError) as e:
            srv.result(j_run)
        assert e.value.status == -11
        with pytest.raises(mocd.MocdError) as e:
            srv.cancel(ids[0])  # finished jobs cannot be cancelled
        assert e.value.status == -1
        for k, (jid, ((rp, ci), kw, G)) in enumerate(zip(ids, jobs)):
            if jid == j_queued:
                continue
            assert srv.state(jid) == (mocd.Server.DONE, 0)
            got, ref = srv.result(jid), _alone(rp, ci, kw, G)
            assert got.best == ref.best and np.array_equal(got.labels, ref.labels)
    finally:
        srv.close()
    cur, _ = mocd.debug_pool_usage()
    assert cur == base  # every job's device memory went back


def test_server_response_ratio_admission_completes_everything():
    """Admission by highest response ratio (policy 1) with one job at a time:
    small jobs overtake a large one, every job finishes with its result equal
    to the job run alone."""
    jobs = _jobs()
    big = synth.lfr_style(20000, 16, 50, 0.3, seed=9)[:2]
    srv = mocd.Server(1 << 34, max_running=1, depth=4)
    srv.start(admission_threads=1, policy=1)
    try:
        j_big = srv.submit(big[0], big[1], mocd.Params(seed=2), 30)
        ids = [srv.submit(rp, ci, mocd.Params(**kw), G) for (rp, ci), kw, G in jobs]
        _drain(srv, [j_big] + ids, 1)
        for jid, ((rp, ci), kw, G) in zip(ids, jobs):
            assert srv.state(jid) == (mocd.Server.DONE, 0)
            got, ref = srv.result(jid), _alone(rp, ci, kw, G)
            assert got.best == ref.best and np.array_equal(got.labels, ref.labels)
        assert srv.state(j_big) == (mocd.Server.DONE, 0)
        got, ref = srv.result(j_big), _alone(big[0], big[1], dict(seed=2), 30)
        assert np.array_equal(got.labels, ref.labels)
    finally:
        srv.close()
