"""The largest graphs the engine takes (n = CFPQ_MAX_NODES = 131072: 4096 words per row, the
widest word summaries, tile lists and extraction scans), on every product path, against the
oracle. Sparse inputs keep the closures small; the matrices are full size."""
import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu

N_MAX = 131072

CASES = [
    ("auto", dict(path=eng.PATH_AUTO)),
    ("gather_jacobi", dict(path=eng.PATH_GATHER, schedule=eng.SCHED_JACOBI)),
    ("tensor_tile_skipping", dict(path=eng.PATH_TENSOR, schedule=eng.SCHED_JACOBI)),
    ("worklist", dict(path=eng.PATH_WORKLIST)),
]


def _local_graph(n, m, seed):
    # two labels; each edge spans at most 64 nodes forward (cyclically), so the matrices are full
    # size but most of their 128 x 128 tiles are empty (the tensor path skips them)
    k = synth.key(seed, 7)
    i = np.arange(m, dtype=np.int64)
    src = synth.uniform_int(k, 3 * i, n)
    lab = synth.uniform_int(k, 3 * i + 1, 2)
    dst = (src + 1 + synth.uniform_int(k, 3 * i + 2, 64)) % n
    return np.stack([src, lab, dst], axis=1)


def _graph():
    # the last node takes part (and the cyclic edges join it to node 0)
    e = _local_graph(N_MAX, 160_000, 31)
    extra = np.array([[N_MAX - 2, 0, N_MAX - 1], [N_MAX - 1, 1, 0], [N_MAX - 1, 0, N_MAX - 1]], dtype=np.int64)
    return synth.Graph(n=N_MAX, edges=np.concatenate([e, extra]), labels=["t0", "t1"], meta={"kind": "test"})


@pytest.fixture(scope="module")
def graph_and_reference():
    graph = _graph()
    text = "S A S1\nS A B\nS1 S B\nA t0\nB t1\n"  # a^k b^k
    return graph, text, oracle.hellings(graph, text)


@pytest.mark.parametrize("name,opts", CASES, ids=[c[0] for c in CASES])
def test_largest_graph_every_path(graph_and_reference, name, opts):
    graph, text, ref = graph_and_reference
    g = eng.Grammar(text, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, timeout_s=300.0, **opts)
    q.solve()
    for nm in g.names:
        assert np.array_equal(q.get(nm), ref.pairs(nm)), nm
    all_t = q.triples_all()
    assert all_t.shape[0] == sum(ref.count(a) for a in range(len(g.names)))
    q.close()


def test_one_below_the_largest_graph():
    # n = 131071: the last row word and the last tile are ragged
    n = N_MAX - 1
    g = synth.Graph(n=n, edges=_local_graph(n, 200_000, 32), labels=["t0", "t1"], meta={"kind": "test"})
    text = "S A B\nA t0\nB t1\n"
    gr = eng.Grammar(text, g.labels)
    ref = oracle.hellings(g, text)
    for opts in (dict(path=eng.PATH_AUTO), dict(path=eng.PATH_TENSOR, schedule=eng.SCHED_JACOBI)):
        q = eng.Query(gr, g.n, g.edges, timeout_s=300.0, **opts)
        q.solve()
        assert np.array_equal(q.get("S"), ref.pairs("S"))
        q.close()
