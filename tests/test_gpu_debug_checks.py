"""The debug build (bounds checks that record failures instead of faulting)
on valid inputs: the same results as the oracle, and no failure recorded;
the normal build reports that it checks nothing."""
import numpy as np
import pytest

import oracle
import paper_2506_01752_gb300 as mocd
import synth
from paper_2506_01752_gb300 import build as cuda_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def debug_lib():
    mocd.load()
    lib = mocd.load_library(cuda_build.build(debug=True))
    old = mocd.use_library(lib)
    yield lib
    mocd.use_library(old)


def _ladder():
    u, v, base = [], [], 0
    for d in (5, 20, 40, 100, 300, 600):  # every vote path, hub table included
        u += [base] * d
        v += list(range(base + 1, base + 1 + d))
        base += d + 1
    return synth.csr_from_edges(base, u, v)


@pytest.mark.parametrize("gname,kw", [
    ("lfr-3k", dict(pop_size=64, seed=4)),
    ("ladder", dict(pop_size=40, p_mutation=1.0, seed=5)),
])
def test_debug_build_matches_oracle_without_failures(debug_lib, gname, kw):
    rp, ci = synth.lfr_style(3000, 20, 50, 0.3, seed=2)[:2] if gname == "lfr-3k" else _ladder()
    assert mocd.debug_checks(reset=True)[0]  # the checks are compiled in
    gp, op = mocd.Params(**kw), oracle.Params(**kw)
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, gp)
        mocd.generation(h, 3)
        labels, k1, k2, gen = mocd.get_population(h)
        lab = synth.random_labels(rp.size - 1, 5, seed=1)
        gi, gs = mocd.evaluate(h, lab)
    finally:
        mocd.destroy(h)
    ref = oracle.run(rp, ci, op, oracle.population_init(rp, ci, op), 3)
    assert gen == 3 and np.array_equal(labels, ref.labels)
    assert np.array_equal(k1, ref.k1) and np.array_equal(k2, ref.k2)
    oi, os_ = oracle.objectives(rp, ci, lab)
    assert np.array_equal(gi, oi) and np.array_equal(gs, os_)
    assert mocd.debug_checks() == (True, 0, 0, 0)


def test_normal_build_checks_nothing():
    lib = mocd.load_library(cuda_build.build())
    old = mocd.use_library(lib)
    try:
        assert mocd.debug_checks() == (False, 0, 0, 0)
    finally:
        mocd.use_library(old)
