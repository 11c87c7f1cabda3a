"""The seeded input generators shared by the oracle and the engine's tests and benchmark
(cfpq_synth): the counter-based generator against its published reference outputs, and the
workload recipes (class hierarchy, batched queries, Poisson arrivals) against their stated
structure. CPU only."""
import math

import numpy as np
import pytest

import cfpq_synth as synth


def test_splitmix64_reference_outputs():
    # SplitMix64 (Steele, Lea and Flood, 2014) from state 0: the first four outputs of the
    # reference implementation (state += 0x9E3779B97F4A7C15, then the two multiply-xorshift
    # rounds); u64(k, i) is output number i from state k
    got = [int(x) for x in synth.u64(np.uint64(0), np.arange(4))]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_uniform_int_stays_in_range_and_covers_it():
    k = synth.key(5, 9)
    m = np.array([1, 2, 3, 7, 1000])
    v = synth.uniform_int(k, np.arange(5 * 4000).reshape(4000, 5), m)
    assert (v >= 0).all() and (v < m).all()
    assert all(len(np.unique(v[:, j])) == m[j] for j in range(4))  # every value of small ranges occurs
    u = synth.uniform01(k, np.arange(200_000))
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005


@pytest.mark.parametrize("n,C,seed", [(2000, 600, 3), (300, 1, 0), (64, 64, 1)])
def test_hierarchy_recipe(n, C, seed):
    g = synth.hierarchy(n, C, seed=seed)
    assert g.n == n and g.labels == ["sc", "sc_r", "ty", "ty_r"]
    e = g.edges
    sc, scr, ty, tyr = (e[e[:, 1] == lab] for lab in range(4))
    # every class c >= 1 has exactly one subClassOf edge, to an earlier class
    assert sorted(sc[:, 0].tolist()) == list(range(1, C))
    assert (sc[:, 2] < sc[:, 0]).all() and (sc[:, 2] >= 0).all()
    # every instance has 1..3 type edges to classes
    assert ((ty[:, 0] >= C) & (ty[:, 0] < n)).all() and ((ty[:, 2] >= 0) & (ty[:, 2] < C)).all()
    per = np.bincount(ty[:, 0] - C, minlength=n - C) if n > C else np.zeros(0, dtype=np.int64)
    assert ((per >= 1) & (per <= 3)).all()
    # every edge is accompanied by its reverse with the _r label
    for fwd, rev in ((sc, scr), (ty, tyr)):
        assert sorted(map(tuple, fwd[:, [0, 2]].tolist())) == sorted(map(tuple, rev[:, [2, 0]].tolist()))
    # seeded: the same seed gives the same graph, another seed another one
    assert np.array_equal(synth.hierarchy(n, C, seed=seed).edges, e)
    if C > 2:
        assert not np.array_equal(synth.hierarchy(n, C, seed=seed + 1).edges, e)


def test_batch_queries_recipe():
    qs = synth.batch_queries(64, seed=0)
    assert len(qs) == 64
    ns = [g.n for g, _ in qs]
    assert min(ns) >= 64 and max(ns) <= 4096
    assert max(ns) > 1000 and min(ns) < 300  # log-uniform: both ends of the range are drawn
    for g, gram in qs:
        assert g.meta["n_classes"] == max(1, int(round(0.3 * g.n)))
        assert gram in (synth.GRAMMAR_Q1, synth.GRAMMAR_QSC)
    assert {gram for _, gram in qs} == {synth.GRAMMAR_Q1, synth.GRAMMAR_QSC}


def test_poisson_arrivals_rate():
    t = synth.poisson_arrivals(20_000, 500.0, seed=2)
    assert (np.diff(t) > 0).all() and t[0] > 0
    # mean gap 1 / rate, within a few standard errors (the gaps are exponential)
    gap = float(t[-1]) / len(t)
    assert abs(gap - 1.0 / 500.0) < 4.0 * (1.0 / 500.0) / math.sqrt(len(t))


def test_communities_recipe():
    # every node has `degree` out-edges, all inside its own community of about n / k nodes
    n, k, d = 3000, 7, 3
    g = synth.communities(n, k, d, seed=2)
    e = np.asarray(g.edges, dtype=np.int64)
    assert e.shape == (n * d, 3) and (e[:, 1] == 0).all()
    assert (np.bincount(e[:, 0], minlength=n) == d).all()
    assert (e[:, 0] * k // n == e[:, 2] * k // n).all()
    sizes = np.bincount(np.arange(n) * k // n)
    assert sizes.max() - sizes.min() <= 1
    again = synth.communities(n, k, d, seed=2)
    assert np.array_equal(again.edges, g.edges)
