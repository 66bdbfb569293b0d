"""Error paths exercised by host-side failure injection (no GPU fault is
ever provoked): a device allocation that fails leaves the context usable and
the next call succeeds with the same results; a generation that cannot be
issued fails its server job instead of returning a short run as a success;
the server's per-job footprint bounds what a job really takes from the
device memory pool."""
import numpy as np
import pytest

import oracle
import paper_2506_01752_gb300 as mocd
import synth

pytestmark = pytest.mark.gpu

OOM = -6


@pytest.fixture(autouse=True)
def disarm():
    mocd.build.build()
    mocd.load()
    yield
    mocd.debug_inject(mocd.SITE_DEVICE_ALLOC, 0, 0, 0)
    mocd.debug_inject(mocd.SITE_GENERATION, 0, 0, 0)


def _graph():
    return synth.lfr_style(3000, 16, 50, 0.3, seed=8)[:2]


def test_upload_allocation_failures():
    """Every allocation of mocd_graph_upload failing in turn: OUT_OF_MEMORY,
    no context; afterwards an upload succeeds."""
    rp, ci = _graph()
    # CSR row pointers, adjacency, node order, the evaluation's oriented row
    # pointers and adjacency, symmetry flag
    for k in range(6):
        mocd.debug_inject(mocd.SITE_DEVICE_ALLOC, k, 1)
        with pytest.raises(mocd.MocdError) as e:
            mocd.graph_upload(rp, ci)
        assert e.value.status == OOM
    mocd.debug_inject(mocd.SITE_DEVICE_ALLOC, 6, 1)  # a seventh allocation would fail: there is none
    mocd.destroy(mocd.graph_upload(rp, ci))


def test_init_and_front_stats_allocation_failures_leave_the_context_usable():
    rp, ci = _graph()
    params, op = mocd.Params(pop_size=40, seed=4), oracle.Params(pop_size=40, seed=4)
    h = mocd.graph_upload(rp, ci)
    try:
        failed = 0
        for k in range(8):
            mocd.debug_inject(mocd.SITE_DEVICE_ALLOC, k, 1)
            try:
                mocd.population_init(h, params)
            except mocd.MocdError as e:
                assert e.status == OOM
                failed += 1
            mocd.debug_inject(mocd.SITE_DEVICE_ALLOC, 0, 0, 0)
        assert failed >= 1
        mocd.population_init(h, params)
        mocd.generation(h, 3)
        ref = oracle.run(rp, ci, op, oracle.population_init(rp, ci, op), 3)
        labels, k1, k2, gen = mocd.get_population(h)
        assert gen == 3 and np.array_equal(labels, ref.labels) and np.array_equal(k1, ref.k1)
        # front statistics: its scratch allocations fail, then succeed
        mocd.debug_inject(mocd.SITE_DEVICE_ALLOC, 0, 1)
        with pytest.raises(mocd.MocdError) as e:
            mocd.front_stats(h)
        assert e.value.status == OOM
        mocd.debug_inject(mocd.SITE_DEVICE_ALLOC, 0, 0, 0)
        st = mocd.front_stats(h)
        fr = mocd.pareto_front(h)
        k, sq, mean, mx = oracle.community_stats(rp, ci, fr.labels)
        assert np.array_equal(st.communities, k) and np.array_equal(st.size_sumsq, sq)
        # the run goes on where it was
        mocd.generation(h, 1)
        ref = oracle.run(rp, ci, op, ref, 1)
        assert np.array_equal(mocd.get_population(h)[0], ref.labels)
    finally:
        mocd.destroy(h)


def test_injected_generation_failure_fails_the_server_job():
    rp, ci = _graph()
    srv = mocd.Server(1 << 34, max_running=2, depth=2)
    try:
        j_fail = srv.submit(rp, ci, mocd.Params(pop_size=16, seed=1), 6)
        # the job's first issue of generations fails
        mocd.debug_inject(mocd.SITE_GENERATION, 0, 1, -8)
        import time
        t_end = time.time() + 60
        while srv.state(j_fail)[0] < mocd.Server.DONE:
            assert time.time() < t_end
            srv.step()
        assert srv.state(j_fail) == (mocd.Server.FAILED, -8)
        with pytest.raises(mocd.MocdError) as e:
            srv.result(j_fail)
        assert e.value.status == -8
        # a later job on the same server runs normally
        j_ok = srv.submit(rp, ci, mocd.Params(pop_size=16, seed=1), 6)
        while srv.state(j_ok)[0] < mocd.Server.DONE:
            assert time.time() < t_end
            srv.step()
        assert srv.state(j_ok) == (mocd.Server.DONE, 0)
    finally:
        srv.close()


@pytest.mark.parametrize("pop", [100, 37])
def test_job_footprint_bounds_the_pool_peak(pop):
    """A whole job alone (upload, init, generations, front download) takes no
    more from the device pool than the footprint the server admits it by,
    give or take the pool's rounding of each of the job's dozen allocations
    (at most one 2 MiB granule each)."""
    rp, ci = synth.lfr_style(100_000, 16, 60, 0.3, seed=9)[:2]
    n, nnz = rp.size - 1, int(rp[-1])
    cur0, _ = mocd.debug_pool_usage(reset_peak=True)
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, mocd.Params(pop_size=pop))
        mocd.generation(h, 4)
        mocd.pareto_front(h)
        mocd.synchronize(h)
    finally:
        mocd.destroy(h)
    _, peak = mocd.debug_pool_usage()
    fp = mocd.job_footprint(rp, pop)
    assert 0 < peak - cur0 <= fp + 16 * (2 << 20), (peak - cur0, fp)
    assert peak - cur0 >= 0.8 * fp, (peak - cur0, fp)  # and the estimate is not loose


def test_pool_keeps_freed_memory_until_trimmed():
    """A destroyed context's memory stays reserved in the library's pool (the
    next context reuses it without mapping fresh memory); mocd_pool_trim
    gives it back to the device."""
    torch = pytest.importorskip("torch")
    rp, ci = synth.lfr_style(100_000, 16, 60, 0.3, seed=9)[:2]
    fp = mocd.job_footprint(rp, 100)
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, mocd.Params())
        mocd.generation(h, 1)
        mocd.synchronize(h)
    finally:
        mocd.destroy(h)
    torch.cuda.synchronize()
    cur, _ = mocd.debug_pool_usage()
    held = torch.cuda.mem_get_info()[0]
    mocd.pool_trim(0)
    freed = torch.cuda.mem_get_info()[0] - held
    assert freed >= 0.5 * fp, (freed, fp)
    assert mocd.debug_pool_usage()[0] == cur  # trimming releases only unused memory
    # and the pool serves the next context as before
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, mocd.Params())
        mocd.generation(h, 1)
        mocd.synchronize(h)
    finally:
        mocd.destroy(h)
    with pytest.raises(mocd.MocdError):
        mocd.pool_trim(-1)
