"""AUTO path: each production group takes, in every loop execution, the cheaper of the
tensor-core product and the CUDA-core gather (chosen on the device). Results equal the
oracle's; every (production, execution) is computed by exactly one of the two kinds."""
import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu


def auto_parity(graph, text, **kw):
    kw.setdefault("timeout_s", 120.0)
    g = eng.Grammar(text, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_AUTO, **kw)
    q.solve()
    ref = oracle.hellings(graph, text)
    for nm in g.names:
        got, exp = q.get(nm), ref.pairs(nm)
        assert got.shape == exp.shape and np.array_equal(got, exp), \
            f"{nm}: engine {got.shape[0]} pairs, oracle {exp.shape[0]}"
    return g, q, q.stats()


def products_each_once(s, text, graph):
    """tensor + gather products = distinct productions x loop executions (the last one included)."""
    cnf = eng.Grammar(text, graph.labels).cnf.contents
    n_bin = len({(cnf.binary[i].lhs, cnf.binary[i].b, cnf.binary[i].c) for i in range(cnf.n_binary)})
    assert s["tensor_products"] + s["gather_products"] == n_bin * s["iterations"]


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("n", [1100, 2600])
def test_dense_closure_picks_tensor(n, use_graph):
    # one dense transitive closure: early executions have large deltas (tensor), the last
    # ones almost none (gather)
    graph = synth.random_graph(n, int(1.6 * n), 1, seed=n)
    _, q, s = auto_parity(graph, "S S S\nS t0\n", use_graph=use_graph)
    assert s["tensor_products"] > 0
    products_each_once(s, "S S S\nS t0\n", graph)


@pytest.mark.parametrize("use_graph", [True, False])
def test_tensor_and_gather_groups_in_one_execution(use_graph):
    # two independent closures: S over a dense random relation (its early executions take the
    # tensor cores) and A over a short chain (its deltas stay tiny: always the gather), so the
    # same executions run both kinds; the gather must still do A's listed items while it skips
    # S's
    n = 1100
    dense = synth.random_graph(n, int(1.6 * n), 1, seed=7).edges
    chain = np.array([[i, 1, i + 1] for i in range(40, 52)], dtype=np.int64)
    graph = synth.Graph(n=n, edges=np.concatenate([dense, chain]), labels=["t0", "t1"], meta={"kind": "test"})
    text = "S S S\nS t0\nA A A\nA t1\n"
    _, q, s = auto_parity(graph, text, use_graph=use_graph)
    assert s["tensor_products"] > 0 and s["gather_products"] > 0
    products_each_once(s, text, graph)


@pytest.mark.parametrize("use_graph", [True, False])
def test_sparse_hierarchy_mixed(use_graph):
    graph = synth.hierarchy(4096, 1200, seed=4)
    _, q, s = auto_parity(graph, synth.GRAMMAR_Q1, use_graph=use_graph)
    products_each_once(s, synth.GRAMMAR_Q1, graph)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("schedule", [eng.SCHED_INPLACE, eng.SCHED_JACOBI])
def test_random_grammars(seed, schedule):
    graph = synth.random_graph(150 + 120 * seed, 900 + 700 * seed, 3, seed=seed)
    text = synth.random_grammar_text(5, 3, 9, 6, seed % 3, seed=seed)
    _, q, s = auto_parity(graph, text, schedule=schedule)
    products_each_once(s, text, graph)


def test_jacobi_loop_count_matches_algorithm1():
    # whichever kind computes a product, a Jacobi execution is one application of the
    # loop body: the loop count is Algorithm 1's
    graph = synth.random_graph(1500, 2400, 1, seed=3)
    text = "S S S\nS t0\n"
    _, q, s = auto_parity(graph, text, schedule=eng.SCHED_JACOBI)
    _, _, k = oracle.matrix_closure_sparse(graph, text)
    assert s["iterations"] == k


def same_depth_pairs(graph):
    parent = {int(s): int(d) for s, l, d in graph.edges if l == 0}
    C = graph.meta["n_classes"]
    depth = np.zeros(C, dtype=np.int64)
    for c in range(1, C):
        depth[c] = depth[parent[c]] + 1
    sizes = np.bincount(depth)
    return int((sizes[1:] ** 2).sum())


@pytest.mark.parametrize("path", [eng.PATH_AUTO, eng.PATH_TENSOR, eng.PATH_GATHER])
def test_same_generation_4096(path):
    graph = synth.hierarchy(4096, 1200, seed=2)
    g = eng.Grammar(synth.GRAMMAR_SG, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=path, timeout_s=120.0)
    q.solve()
    ref = oracle.hellings(graph, synth.GRAMMAR_SG)
    for nm in g.names:
        assert np.array_equal(q.get(nm), ref.pairs(nm)), nm


def test_same_generation_full_size():
    # n = 16384, 5000 classes: |R_S| = sum over depths >= 1 of (classes at that depth)^2, and
    # the Jacobi loop count is the oracle's sparse Algorithm 1 count
    graph = synth.hierarchy(16384, 5000, seed=0)
    g = eng.Grammar(synth.GRAMMAR_SG, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_AUTO, schedule=eng.SCHED_JACOBI, timeout_s=300.0)
    q.solve()
    assert q.count("S") == same_depth_pairs(graph)
    _, _, k = oracle.matrix_closure_sparse(graph, synth.GRAMMAR_SG)
    s = q.stats()
    assert s["iterations"] == k
    products_each_once(s, synth.GRAMMAR_SG, graph)


def test_long_chain_hands_over_to_the_worklist():
    # two cycles: every loop execution adds about one pair; after a long run of such
    # executions the automatic path stops the matrix loop and the worklist path finishes the
    # closure from the current delta
    graph = synth.two_cycles(64, 63)
    g = eng.Grammar(synth.GRAMMAR_C3, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_AUTO)
    q.solve()
    s = q.stats()
    assert s["worklist_items"] > 0 and 64 <= s["iterations"] < 64 * 63
    ref = oracle.hellings(graph, synth.GRAMMAR_C3)
    for nm in g.names:
        assert np.array_equal(q.get(nm), ref.pairs(nm)), nm
    # under Jacobi the loop keeps Algorithm 1's exact count, so it never hands over
    qj = eng.Query(g, graph.n, graph.edges, path=eng.PATH_AUTO, schedule=eng.SCHED_JACOBI, timeout_s=120.0)
    qj.solve()
    assert qj.stats()["worklist_items"] == 0 and qj.stats()["iterations"] == 2 * 64 * 63 + 1


def test_long_chain_full_size_automatic():
    p, qq = 4096, 4095
    graph = synth.two_cycles(p, qq)
    g = eng.Grammar(synth.GRAMMAR_C3, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_AUTO, timeout_s=300.0)
    q.solve()
    assert q.stats()["worklist_items"] > 0
    assert q.count("S") == p * qq and q.count("S1") == p * qq


@pytest.fixture(scope="module")
def block_diagonal():
    graph = synth.communities(16384, 32, 2, seed=3)
    text = "S S S\nS t0\n"
    return graph, text, oracle.hellings(graph, text).pairs("S")


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("kind", [eng.TENSOR_FP4, eng.TENSOR_FP8], ids=["fp4", "fp8"])
def test_block_diagonal_closure_prices_tile_skipping(block_diagonal, use_graph, kind):
    """A transitive closure over 32 communities of 512 nodes (block-diagonal matrices): once
    the gather has grown expensive, the cost model asks for the tile counts and then prices a
    tensor product by its live K steps, which are a small fraction of the dense product here.
    Some executions must run on the tensor cores with tile skipping (executed work far below
    the dense product), and the result must equal the oracle's."""
    graph, text, ref = block_diagonal
    g = eng.Grammar(text, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_AUTO, use_graph=use_graph, tensor_kind=kind,
                  timeout_s=120.0)
    q.solve()
    assert np.array_equal(q.get("S"), ref)
    s = q.stats()
    products_each_once(s, text, graph)
    assert s["tensor_products"] > 0
    assert 0 < s["tensor_live_ops"] < 0.05 * s["dense_ops"]


def test_block_diagonal_closure_default_path_beats_gather_only():
    # the same closure (64 communities, n = 32768): the automatic path against the gather alone
    graph = synth.communities(32768, 64, 2, seed=4)
    text = "S S S\nS t0\n"
    g = eng.Grammar(text, graph.labels)
    times = {}
    for name, path in (("auto", eng.PATH_AUTO), ("gather", eng.PATH_GATHER)):
        q = eng.Query(g, graph.n, graph.edges, path=path, timeout_s=120.0)
        q.solve()
        ts = []
        for _ in range(3):
            q.solve()
            ts.append(q.stats()["solve_ms"])
        times[name] = min(ts)
        if name == "auto":
            assert q.stats()["tensor_products"] > 0
            res = q.get("S")
        else:
            assert np.array_equal(q.get("S"), res)
    assert times["auto"] < times["gather"], times
