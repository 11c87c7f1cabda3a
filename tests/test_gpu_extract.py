"""Extraction of every relation (Algorithm 1's result R_A for all A, Theorem 2) through the
Python binding: the solve's pair counters (seed pairs, and pairs the products added, each
counted when its bit is first set) equal the number of triples on every path, so they size
the buffer of triples_all; when they do not (stale or too small), the exact count from the
first call sizes a second one. Results are compared with the oracle."""
import ctypes

import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu

PATHS = [
    ("auto", dict(path=eng.PATH_AUTO)),
    ("gather-jacobi", dict(path=eng.PATH_GATHER, schedule=eng.SCHED_JACOBI)),
    ("gather-inplace", dict(path=eng.PATH_GATHER, schedule=eng.SCHED_INPLACE)),
    ("tensor-dense", dict(path=eng.PATH_TENSOR, schedule=eng.SCHED_JACOBI, dense_tensor=True)),
    ("tensor-skip", dict(path=eng.PATH_TENSOR, schedule=eng.SCHED_JACOBI)),
    ("worklist", dict(path=eng.PATH_WORKLIST)),
]


def expected_triples(graph, text, names):
    ref = oracle.hellings(graph, text)
    rows = []
    for a, nm in enumerate(names):
        p = ref.pairs(nm)
        rows.append(np.concatenate([np.full((p.shape[0], 1), a, dtype=np.int64), p.astype(np.int64)], axis=1))
    return np.concatenate(rows, axis=0)


@pytest.mark.parametrize("name,opts", PATHS, ids=[p[0] for p in PATHS])
def test_counters_size_the_extraction(name, opts):
    graph = synth.hierarchy(1100, 330, seed=7)
    g = eng.Grammar(synth.GRAMMAR_Q1, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, timeout_s=120.0, **opts)
    q.solve()
    st = q.stats()
    got = q.triples_all()
    assert got.dtype == np.uint32 and got.shape[1] == 3
    assert st["seed_bits"] + st["new_bits"] == got.shape[0]
    assert np.array_equal(got, expected_triples(graph, synth.GRAMMAR_Q1, g.names))
    q.close()


def test_counters_after_a_hand_over():
    # the automatic path ends this closure on the worklist path; the worklist counts the
    # pairs it adds like the loop's products
    graph = synth.two_cycles(40, 39)
    g = eng.Grammar(synth.GRAMMAR_C3, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, timeout_s=120.0)
    q.solve()
    st = q.stats()
    assert st["worklist_items"] > 0
    got = q.triples_all()
    assert st["seed_bits"] + st["new_bits"] == got.shape[0]
    assert np.array_equal(got, expected_triples(graph, synth.GRAMMAR_C3, g.names))
    q.close()


def test_too_small_a_hint_falls_back_to_the_exact_count(monkeypatch):
    graph = synth.hierarchy(900, 250, seed=2)
    g = eng.Grammar(synth.GRAMMAR_Q1, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, timeout_s=120.0)
    q.solve()
    ref = q.triples_all()
    lib = eng._lib()
    real = lib.cfpq_stats_get

    def understated(h, p):
        rc = real(h, p)
        p._obj.seed_bits, p._obj.new_bits = 1, 0  # a hint of one triple
        return rc

    monkeypatch.setattr(lib, "cfpq_stats_get", understated)
    got = q.triples_all()
    monkeypatch.undo()
    assert ref.shape[0] > 1 and np.array_equal(got, ref)
    q.close()


def test_results_survive_the_next_extraction():
    # each call returns its own buffer: a later extraction does not overwrite an earlier result
    graph = synth.hierarchy(900, 250, seed=3)
    g = eng.Grammar(synth.GRAMMAR_Q1, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, timeout_s=120.0)
    q.solve()
    first = q.triples_all()
    keep = first.copy()
    per = [q.triples(nm) for nm in g.names]
    second = q.triples_all()
    assert np.array_equal(first, keep) and np.array_equal(second, keep)
    assert np.array_equal(np.concatenate(per, axis=0), keep)
    assert ctypes.sizeof(eng.Triple) == 12
    q.close()


def test_concurrent_solves_on_two_streams():
    """Two contexts solved at the same time from two host threads on two streams: each
    launches the persistent gather loop (a cooperative grid over the whole device), so the
    launches share the GPU; both closures equal the oracle's."""
    import threading

    import torch

    cases = []
    for seed, text in ((21, synth.GRAMMAR_Q1), (22, synth.GRAMMAR_QSC)):
        graph = synth.hierarchy(6000, 1800, seed=seed)
        g = eng.Grammar(text, graph.labels)
        cases.append((graph, text, g, eng.Query(g, graph.n, graph.edges, path=eng.PATH_GATHER, timeout_s=120.0)))
    streams = [torch.cuda.Stream() for _ in cases]
    errors = []

    def work(q, s):
        try:
            for _ in range(4):
                q.solve(s)
        except Exception as e:  # reported below, on the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(c[3], s)) for c, s in zip(cases, streams)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    for graph, text, g, q in cases:
        assert np.array_equal(q.triples_all(), expected_triples(graph, text, g.names))
        q.close()
