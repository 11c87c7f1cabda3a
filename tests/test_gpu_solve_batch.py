"""Batched closure (one grouped persistent launch): every query's result equals its
oracle result and its result when solved alone (per-query convergence)."""
import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu


def _mk(graph, text, **kw):
    g = eng.Grammar(text, graph.labels)
    return g, eng.Query(g, graph.n, graph.edges, path=eng.PATH_GATHER, **kw)


def test_batch_small_mixed_schedules():
    qs = []
    for j in range(12):
        graph = synth.random_graph(30 + 11 * j, 80 + 9 * j, 2, seed=j)
        text = synth.random_grammar_text(4, 2, 7, 5, j % 2, seed=j)
        qs.append((graph, text) + _mk(graph, text, schedule=j % 2))
    eng.solve_batch([q for _, _, _, q in qs])
    for graph, text, g, q in qs:
        ref = oracle.hellings(graph, text)
        for nm in g.names:
            assert np.array_equal(q.get(nm), ref.pairs(nm)), nm


def test_batch_jacobi_iteration_counts():
    qs = [(p, qq) + _mk(synth.two_cycles(p, qq), synth.GRAMMAR_C3, schedule=eng.SCHED_JACOBI)
          for p, qq in [(2, 1), (3, 2), (5, 4), (7, 3)]]
    eng.solve_batch([q for *_, q in qs])
    for p, qq, g, q in qs:
        assert q.stats()["iterations"] == 2 * p * qq + 1


def test_batch_256_hierarchy_alone_vs_mixed():
    work = synth.batch_queries(256, 64, 4096, 0.3, seed=0)
    mixed = [_mk(graph, text) for graph, text in work]
    eng.solve_batch([q for _, q in mixed])
    for idx, ((graph, text), (g, q)) in enumerate(zip(work, mixed)):
        ref = oracle.hellings(graph, text)
        for nm in g.names:
            assert np.array_equal(q.get(nm), ref.pairs(nm)), (idx, nm)
    # alone: a sample solved one at a time gives the same sets (the in-place iteration count
    # depends on the order the production groups run in, so it is not compared here)
    for idx in range(0, 256, 37):
        graph, text = work[idx]
        g, q = _mk(graph, text)
        q.solve()
        _, qm = mixed[idx]
        for nm in g.names:
            assert np.array_equal(q.get(nm), qm.get(nm))


def test_batch_jacobi_alone_vs_mixed_iterations():
    # under the Jacobi schedule every query runs exactly Algorithm 1's loop count, alone or mixed
    work = synth.batch_queries(48, 64, 2048, 0.3, seed=3)
    mixed = [_mk(graph, text, schedule=eng.SCHED_JACOBI) for graph, text in work]
    eng.solve_batch([q for _, q in mixed])
    for (graph, text), (g, qm) in zip(work, mixed):
        ga, qa = _mk(graph, text, schedule=eng.SCHED_JACOBI)
        qa.solve()
        assert qa.stats()["iterations"] == qm.stats()["iterations"]
        ref = oracle.hellings(graph, text)
        for nm in g.names:
            assert np.array_equal(qm.get(nm), ref.pairs(nm))


def test_batch_iteration_limit_is_per_query():
    a = _mk(synth.two_cycles(9, 8), synth.GRAMMAR_C3, max_iter=4)
    graph = synth.hierarchy(500, 150, seed=1)
    b = _mk(graph, synth.GRAMMAR_Q1)
    assert eng.solve_batch([a[1], b[1]], check=False) == eng.ERR_ITER_LIMIT
    assert a[1].stats()["iterations"] == 4
    ref = oracle.hellings(graph, synth.GRAMMAR_Q1)
    for nm in b[0].names:
        assert np.array_equal(b[1].get(nm), ref.pairs(nm))


def test_batch_wall_clock_limit_is_checked_on_the_device():
    # two cycles 64/63 need 2pq+1 = 8065 Jacobi rounds; a 2 ms limit ends the launch early with
    # TIMEOUT, the contexts stay unsolved, and the same contexts solve normally afterwards
    graph = synth.two_cycles(64, 63)
    g = eng.Grammar(synth.GRAMMAR_C3, graph.labels)
    slow = eng.Query(g, graph.n, graph.edges, path=eng.PATH_GATHER, schedule=eng.SCHED_JACOBI, timeout_s=0.002)
    other = eng.Query(g, graph.n, graph.edges, path=eng.PATH_GATHER)
    assert eng.solve_batch([slow, other], check=False) == eng.ERR_TIMEOUT
    with pytest.raises(eng.CfpqError):
        other.count("S")
    fresh = eng.Query(g, graph.n, graph.edges, path=eng.PATH_GATHER, schedule=eng.SCHED_JACOBI)
    eng.solve_batch([fresh, other])
    assert fresh.count("S") == 64 * 63 and other.count("S") == 64 * 63
    assert fresh.stats()["iterations"] == 2 * 64 * 63 + 1
