"""Batched generations (several instances, one CUDA-graph launch per
generation): every instance must evolve exactly as it does alone, which the
oracle pins."""
import numpy as np
import pytest

import oracle
import paper_2506_01752_gb300 as mocd
import synth
from _golden import graph, load

pytestmark = pytest.mark.gpu


def _instances():
    return [
        (synth.workload("planted-1k", seed=0)[:2], dict(pop_size=100, seed=1)),
        (synth.lfr_style(3000, 20, 50, 0.3, seed=2)[:2], dict(pop_size=64, seed=2)),
        (graph(load("appE_operator_example.txt")), dict(pop_size=8, n_parents=3, seed=3)),
        (synth.lfr_style(1500, 12, 60, 0.4, seed=4)[:2], dict(pop_size=100, seed=4, p_mutation=0.5)),
        (graph(load("fig2_toy_graph.txt")), dict(pop_size=33, n_parents=5, seed=5)),
    ]


def _run(autotune, merged=None):
    inst = _instances()
    ctxs = [mocd.graph_upload(rp, ci) for (rp, ci), _ in inst]
    try:
        for c, (_, kw) in zip(ctxs, inst):
            mocd.population_init(c, mocd.Params(**kw))
        b = mocd.batch_create(ctxs)
        try:
            if autotune:
                shape = mocd.batch_autotune(b, 2)
                assert shape in (1, 2, 4, 8, 16)
                mocd.batch_synchronize(b)
                # the members advanced during tuning: start them again
                for c, (_, kw) in zip(ctxs, inst):
                    mocd.population_init(c, mocd.Params(**kw))
                with pytest.raises(mocd.MocdError) as e:
                    mocd.batch_generation(b, 1)
                assert e.value.status == -9
                mocd.batch_destroy(b)
                b = mocd.batch_create(ctxs)
            if merged is not None:
                mocd.batch_configure(b, 2, merged)
                assert mocd.batch_form(b) == (2, merged)
                with pytest.raises(mocd.MocdError):
                    mocd.batch_configure(b, 2, 3)
            mocd.batch_generation(b, 4)
            mocd.batch_synchronize(b)
            for c, ((rp, ci), kw) in zip(ctxs, inst):
                op = oracle.Params(**kw)
                ref = oracle.run(rp, ci, op, oracle.population_init(rp, ci, op), 4)
                labels, k1, k2, gen = mocd.get_population(c)
                assert gen == 4
                assert np.array_equal(k1, ref.k1) and np.array_equal(k2, ref.k2)
                assert np.array_equal(labels, ref.labels)
            # a member keeps working on its own after batch generations
            mocd.generation(ctxs[0], 1)
            (rp, ci), kw = inst[0]
            op = oracle.Params(**kw)
            ref = oracle.run(rp, ci, op, oracle.population_init(rp, ci, op), 5)
            assert np.array_equal(mocd.get_population(ctxs[0])[0], ref.labels)
        finally:
            mocd.batch_destroy(b)
    finally:
        for c in ctxs:
            mocd.destroy(c)


def test_batch_matches_oracle():
    _run(autotune=False)


def test_batch_after_autotune_matches_oracle():
    _run(autotune=True)


@pytest.mark.parametrize("form", [0, 1, 2])
def test_batch_forms_match_oracle(form):
    """Per-member chains, the merged multi-population selection and the
    multi-member crossover, vote, evaluation and selection launches give the
    same generations (the oracle's); the members differ in size, N_p and E_S
    (3, 4 and 5: the multi-member crossover takes the general E_S form)."""
    _run(autotune=False, merged=form)


def test_batch_rejects_bad_members():
    rp, ci = graph(load("fig2_toy_graph.txt"))
    c = mocd.graph_upload(rp, ci)
    try:
        with pytest.raises(mocd.MocdError) as e:
            mocd.batch_create([c])  # not initialised
        assert e.value.status == -9
        mocd.population_init(c, mocd.Params(pop_size=10))
        with pytest.raises(mocd.MocdError) as e:
            mocd.batch_create([c, c])  # repeated member
        assert e.value.status == -1
    finally:
        mocd.destroy(c)


def test_full_batch_of_64_sampled_against_oracle():
    """The batched-jobs workload at full size (64 uneven jobs, n from 1e3 to
    5e4, N_p = 100 each, seeds as the benchmark uses them), in the launch shape
    the autotuner picks: two batched generations, then six jobs (the
    smallest, the largest and four in between) compared bit for bit with the
    oracle run of the same job."""
    insts = synth.batch_instances(64, seed=0)
    ctxs = [mocd.graph_upload(rp, ci) for rp, ci, _, _ in insts]
    try:
        for k, c in enumerate(ctxs):
            mocd.population_init(c, mocd.Params(seed=k))
        b = mocd.batch_create(ctxs)
        mocd.batch_autotune(b, 1)
        shape, form = mocd.batch_form(b)
        mocd.batch_destroy(b)
        for k, c in enumerate(ctxs):
            mocd.population_init(c, mocd.Params(seed=k))
        b = mocd.batch_create(ctxs)
        try:
            mocd.batch_configure(b, shape, form)
            mocd.batch_generation(b, 2)
            mocd.batch_synchronize(b)
        finally:
            mocd.batch_destroy(b)
        sizes = np.array([rp.size - 1 for rp, _, _, _ in insts])
        order = np.argsort(sizes)
        sample = sorted({int(order[0]), int(order[-1]), *[int(order[q]) for q in (13, 29, 41, 55)]})
        for k in sample:
            rp, ci, _, _ = insts[k]
            op = oracle.Params(seed=k)
            ref = oracle.run(rp, ci, op, oracle.population_init(rp, ci, op), 2)
            labels, k1, k2, gen = mocd.get_population(ctxs[k])
            assert gen == 2
            assert np.array_equal(k1, ref.k1) and np.array_equal(k2, ref.k2), k
            assert np.array_equal(labels, ref.labels), k
    finally:
        for c in ctxs:
            mocd.destroy(c)
