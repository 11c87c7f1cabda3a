"""Worklist path (semi-naive at the grain of single pairs): the same least
fixpoint as Algorithm 1, against the oracle and the two-cycle closed form at full size."""
import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu


def wl(graph, text, **kw):
    kw.setdefault("timeout_s", 300.0)
    g = eng.Grammar(text, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_WORKLIST, **kw)
    q.solve()
    return g, q


def parity(graph, text):
    g, q = wl(graph, text)
    ref = oracle.hellings(graph, text)
    for nm in g.names:
        assert np.array_equal(q.get(nm), ref.pairs(nm)), nm
    return g, q


def test_worked_example():
    parity(synth.worked_example_graph(), synth.GRAMMAR_WORKED)


@pytest.mark.parametrize("seed", range(6))
def test_random(seed):
    graph = synth.random_graph(40 + 9 * seed, 100 + 15 * seed, 3, seed=seed)
    parity(graph, synth.random_grammar_text(5, 3, 9, 6, seed % 3, seed=seed))


@pytest.mark.parametrize("n", [1, 33, 257, 600])
def test_ragged_and_dense(n):
    parity(synth.random_graph(n, 3 * n, 2, seed=n), "S S S\nS A B\nA t0\nB t1\nE eps\nF E S\n")


@pytest.mark.parametrize("text", [synth.GRAMMAR_Q1, synth.GRAMMAR_QSC, synth.GRAMMAR_Q2])
def test_hierarchy(text):
    parity(synth.hierarchy(3000, 900, seed=6), text)


@pytest.mark.parametrize("p,q", [(6, 4), (9, 6), (33, 32), (128, 127)])
def test_two_cycles(p, q):
    parity(synth.two_cycles(p, q), synth.GRAMMAR_C3)


def test_two_cycles_full_size_closed_form():
    """Two directed cycles of 4096 and 4095 nodes sharing node 0, S -> a S b | a b: since
    gcd = 1, R_S = R_S1 = (a-cycle nodes) x (b-cycle nodes), 16,773,120 pairs each."""
    p, qq = 4096, 4095
    graph = synth.two_cycles(p, qq)
    g, q = wl(graph, synth.GRAMMAR_C3, timeout_s=600.0)
    a_nodes = np.arange(p, dtype=np.uint32)
    b_nodes = np.sort(np.concatenate([[0], np.arange(p, p + qq - 1)]).astype(np.uint32))
    exp = np.stack([np.repeat(a_nodes, qq), np.tile(b_nodes, p)], axis=1)
    for nm in ("S", "S1"):
        got = q.get(nm)
        assert got.shape == (p * qq, 2)
        assert np.array_equal(got, exp), nm
    assert q.count("A") == p and q.count("B") == qq


def labelled_graph(n, edges, labels):
    return synth.Graph(n=n, edges=np.asarray(edges, dtype=np.int64).reshape(-1, 3), labels=list(labels),
                       meta={"kind": "test"})


def test_period_one_chain_is_transitive_closure():
    # S -> S B | B on a directed path: S is the left operand of its own production with the
    # static B as partner (a chain of period 1 moving the column); R_S = all (i, j), i < j
    n = 3000
    graph = labelled_graph(n, [(i, 0, i + 1) for i in range(n - 1)], ["b"])
    text = "S S B\nS b\nB b\n"
    g, q = wl(graph, text)
    assert q.count("S") == n * (n - 1) // 2
    small = labelled_graph(300, [(i, 0, i + 1) for i in range(299)], ["b"])
    parity(small, text)


def test_chain_through_a_branch_and_a_merge():
    # a b-path with a fork (node 700 has two b-successors) and a node of in-degree 2: the
    # chain loses its unique successor at the fork, the general join takes over, and the two
    # branches' chains meet pairs that are already set
    n = 1500
    e = [(i, 0, i + 1) for i in range(n - 1) if i != 1000]
    e += [(700, 0, 1001), (1000, 0, 1200)]
    e += [(i, 1, i) for i in range(0, n, 7)]  # a-loops: S seeds a b* on every seventh node
    graph = labelled_graph(n, e, ["b", "a"])
    parity(graph, "S S B\nS a\nB b\n")


def test_period_two_chain_on_one_coordinate():
    # S -> S1 C, S1 -> S B: both chain steps move the column (b then c), S = a (b c)*
    n = 2401
    e = [(i, 0 if i % 2 == 0 else 1, i + 1) for i in range(n - 1)]  # b, c, b, c, ...
    e += [(i, 2, i) for i in range(0, n, 2)]  # a-loops at the even nodes
    graph = labelled_graph(n, e, ["b", "c", "a"])
    text = "S S1 C\nS1 S B\nS a\nB b\nC c\n"
    g, q = wl(graph, text)
    # (i, j) with i even and j = i + 2k, k >= 0
    assert q.count("S") == sum((n - 1 - i) // 2 + 1 for i in range(0, n, 2))
    parity(labelled_graph(401, e[:400] + [(i, 2, i) for i in range(0, 401, 2)], ["b", "c", "a"]), text)


def test_static_relations_with_repeats_eps_and_empty():
    # the static relations are the seeds as sets: repeated edges, two labels seeding the same
    # pair of B, eps on B (the diagonal, which also meets the a-loops' pairs), and a static Z
    # with no pair at all; n spans several 32-bit words with a ragged tail
    n = 777
    e = [(i, 0, i + 1) for i in range(n - 1)] * 2
    e += [(i, 1, i + 1) for i in range(0, n - 1, 3)]
    e += [(i, 2, i) for i in range(0, n, 5)] * 2
    graph = labelled_graph(n, e, ["b", "c", "a", "z"])
    parity(graph, "S S B\nS a\nB b\nB c\nB eps\nX S Z\nZ z\nY B S\n")


@pytest.mark.parametrize("path", ["auto", "worklist"])
def test_tables_rebuilt_per_context(path):
    # two contexts one after the other: the second's tables come from its own seed, not from
    # the memory the first left behind
    p = eng.PATH_AUTO if path == "auto" else eng.PATH_WORKLIST
    for (pp, qq) in ((40, 39), (33, 32)):
        graph = synth.two_cycles(pp, qq)
        g = eng.Grammar(synth.GRAMMAR_C3, graph.labels)
        q = eng.Query(g, graph.n, graph.edges, path=p, timeout_s=300.0)
        q.solve()
        ref = oracle.hellings(graph, synth.GRAMMAR_C3)
        for nm in g.names:
            assert np.array_equal(q.get(nm), ref.pairs(nm)), (pp, nm)
        assert q.stats()["worklist_items"] > 0  # the automatic path handed over to the worklist
        q.close()
