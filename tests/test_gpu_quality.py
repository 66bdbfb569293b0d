"""Whole-run quality smoke on the CUDA path: G = 100 generations of the
benchmark graph shapes, then the recommended member of the returned front
(Alg. 3) scored against the planted communities. The paper reports NMI near 1
for mixing mu <= 0.3 (Sec. 5); the smoke asks for NMI >= 0.9 there."""
import numpy as np
import pytest

import paper_2506_01752_gb300 as mocd
import synth
from synth import quality

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mocd.build.build()
    mocd.load()


def _recommended(rp, ci, G, **kw):
    h = mocd.graph_upload(rp, ci)
    try:
        mocd.population_init(h, mocd.Params(**kw))
        mocd.generation(h, G)
        fr = mocd.pareto_front(h)
    finally:
        mocd.destroy(h)
    # the front is mutually non-dominated in the integer keys (m - intra, S)
    k1 = int(rp[-1] // 2) - fr.intra.astype(np.int64)
    k2 = fr.sumsq.astype(np.int64)
    for a in range(k1.size):
        dom = (k1 <= k1[a]) & (k2 <= k2[a]) & ((k1 < k1[a]) | (k2 < k2[a]))
        assert not dom.any()
    return fr.labels[fr.best]


@pytest.mark.parametrize("init_mode", [0, 1])
def test_planted_1k_recovers_truth(init_mode):
    rp, ci, truth = synth.workload("planted-1k", seed=0)
    lab = _recommended(rp, ci, 100, seed=0, init_mode=init_mode)
    assert quality.nmi(lab, truth) >= 0.9


@pytest.mark.parametrize("init_mode", [0, 1])
@pytest.mark.parametrize("mu", [0.1, 0.3])
def test_lfr_40k_recovers_truth(mu, init_mode):
    rp, ci, truth = synth.workload("lfr-40k", seed=0, mu=mu)
    lab = _recommended(rp, ci, 100, seed=0, init_mode=init_mode)
    assert quality.nmi(lab, truth) >= 0.9
    assert quality.pairwise_f1(lab, truth) >= 0.5
