"""Device memory of cfpq_create contexts comes from the library's pool: memory a destroyed
context released stays reserved for the next context (no new allocation), cfpq_trim_memory
hands it back to the system, and a context built on reused memory (which holds the previous
context's bits) still computes the closure of Algorithm 1 exactly."""
import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu

MiB = 1 << 20


def _free():
    import torch

    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_destroyed_memory_is_reused_then_trimmed():
    graph = synth.hierarchy(8192, 2500, seed=11)
    g = eng.Grammar(synth.GRAMMAR_Q1, graph.labels)
    eng.trim_memory(0)
    base = _free()
    q = eng.Query(g, graph.n, graph.edges, timeout_s=120.0)
    q.solve()
    ref = q.triples_all()
    held = base - _free()
    assert held > 100 * MiB  # 4 bit planes per non-terminal of 8 MiB each, and the rest
    q.close()
    assert base - _free() >= held - 4 * MiB  # kept in the pool
    q2 = eng.Query(g, graph.n, graph.edges, timeout_s=120.0)
    q2.solve()
    assert base - _free() <= held + 4 * MiB  # the same memory again, nothing new
    assert np.array_equal(q2.triples_all(), ref)
    q2.close()
    eng.trim_memory(0)
    assert base - _free() < 16 * MiB  # handed back


def test_reused_memory_gives_the_oracle_closure():
    """A dense query fills the pool's memory with set bits; the next, sparser query of the
    same size reuses that memory and must not see any of them."""
    dense = synth.random_graph(700, 9000, 1, seed=4)
    qd = eng.Query(eng.Grammar("S S S\nS t0\n", dense.labels), dense.n, dense.edges, timeout_s=120.0)
    qd.solve()
    assert qd.count("S") > 700 * 600
    qd.close()
    graph = synth.hierarchy(700, 200, seed=3)
    g = eng.Grammar(synth.GRAMMAR_Q1, graph.labels)
    for path in (eng.PATH_AUTO, eng.PATH_GATHER, eng.PATH_WORKLIST):
        q = eng.Query(g, graph.n, graph.edges, path=path, timeout_s=120.0)
        q.solve()
        ref = oracle.hellings(graph, synth.GRAMMAR_Q1)
        for nm in g.names:
            assert np.array_equal(q.get(nm), ref.pairs(nm)), (path, nm)
        q.close()


def test_trim_keeps_live_contexts():
    graph = synth.hierarchy(1500, 450, seed=5)
    g = eng.Grammar(synth.GRAMMAR_Q1, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, timeout_s=120.0)
    q.solve()
    before = q.triples_all()
    eng.trim_memory(0)
    q.solve()  # the context's memory is still its own
    assert np.array_equal(q.triples_all(), before)
    q.close()
