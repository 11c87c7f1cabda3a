"""The benchmark's own configuration against the CPU oracle, bit-exact.

bench.py times Algorithm 1 (Section 4.2) with the Jacobi loop body and every Boolean product
on the tensor cores as a dense product (every K step issued, no tile skipping) on the
hierarchy of n = 16384 nodes (5000 classes, seed 0), for Query 1 and the subClassOf-only
query. At that size one CTA runs about 55 output tiles of K = 65,536 in turn, so mbarrier
phases and the accumulator hand-back carry across many tiles; these tests check every
relation of that exact configuration against the oracle (Theorem 2: the closure is R_A), for
each operand format of the tensor products (the default, E4M3 and E2M1)."""
import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu

N, CLASSES, SEED = 16384, 5000, 0


@pytest.fixture(scope="module")
def graph():
    return synth.hierarchy(N, CLASSES, seed=SEED)


@pytest.mark.parametrize("kind", [eng.TENSOR_AUTO, eng.TENSOR_FP8, eng.TENSOR_FP4], ids=["auto", "fp8", "fp4"])
@pytest.mark.parametrize("text", [synth.GRAMMAR_Q1, synth.GRAMMAR_QSC], ids=["Q1", "QSC"])
def test_dense_tensor_jacobi_full_size(graph, text, kind):
    g = eng.Grammar(text, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_TENSOR, schedule=eng.SCHED_JACOBI, dense_tensor=True,
                  timeout_s=300.0, tensor_kind=kind)
    q.solve()
    ref = oracle.hellings(graph, text)
    for nm in g.names:
        got, exp = q.get(nm), ref.pairs(nm)
        assert got.shape == exp.shape and np.array_equal(got, exp), \
            f"{nm}: engine {got.shape[0]} pairs, oracle {exp.shape[0]}"
    s = q.stats()
    # every product of every execution ran on the tensor cores, every K step issued
    nprod = len(set(map(tuple, oracle.parse_grammar(text, graph.labels).binary)))
    _, _, k = oracle.matrix_closure_sparse(graph, text)
    assert s["iterations"] == k
    assert s["tensor_products"] == k * nprod and s["gather_products"] == 0
    assert s["tensor_live_ops"] == s["dense_ops"] == k * nprod * 2.0 * float(N) ** 3


def test_dense_tensor_jacobi_repeat_solves(graph):
    # the timed loop solves the same context again and again: each solve equals the first
    text = synth.GRAMMAR_QSC
    g = eng.Grammar(text, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_TENSOR, schedule=eng.SCHED_JACOBI, dense_tensor=True,
                  timeout_s=300.0)
    ref = oracle.hellings(graph, text)
    for _ in range(3):
        q.solve()
        for nm in g.names:
            assert np.array_equal(q.get(nm), ref.pairs(nm)), nm
