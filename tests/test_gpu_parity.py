"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

The bar is bit-exact: every R_A, as a set of (A, m, n) triples, equals the oracle's."""
import ctypes

import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu


def engine_sets(q, names):
    return {nm: set(map(tuple, q.get(nm).tolist())) for nm in names}


def solve_engine(graph, text, **kw):
    kw.setdefault("timeout_s", 120.0)  # device-side bound on any runaway loop
    g = eng.Grammar(text, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, **kw)
    q.solve()
    return g, q


def assert_parity(graph, text, **kw):
    g, q = solve_engine(graph, text, **kw)
    ref = oracle.hellings(graph, text)
    for nm in g.names:
        got, exp = q.get(nm), ref.pairs(nm)
        assert got.shape == exp.shape and np.array_equal(got, exp), \
            f"{nm}: engine {got.shape[0]} pairs, oracle {exp.shape[0]}"
    return g, q, ref


SCHEDULES = [eng.SCHED_INPLACE, eng.SCHED_JACOBI]


# ------------------------------------------------------------------ worked example

@pytest.mark.parametrize("use_graph", [True, False])
def test_worked_example_relations(use_graph):
    graph = synth.worked_example_graph()
    g, q, _ = assert_parity(graph, synth.GRAMMAR_WORKED, use_graph=use_graph)
    assert set(map(tuple, q.get("S").tolist())) == {(0, 0), (0, 2), (1, 2)}


def test_worked_example_every_iteration_jacobi():
    """Jacobi schedule = Algorithm 1's loop body: after k executions the engine holds T_k,
    and the loop stops after k = 6 executions (Section 4.3)."""
    graph = synth.worked_example_graph()
    cnf, snaps, k = oracle.matrix_closure(graph, synth.GRAMMAR_WORKED)
    g, q = solve_engine(graph, synth.GRAMMAR_WORKED, schedule=eng.SCHED_JACOBI)
    assert q.stats()["iterations"] == k == 6
    for it in range(1, 6):
        gg = eng.Grammar(synth.GRAMMAR_WORKED, graph.labels)
        qq = eng.Query(gg, graph.n, graph.edges, schedule=eng.SCHED_JACOBI, max_iter=it)
        assert qq.solve(check=False) == eng.ERR_ITER_LIMIT
        for a, nm in enumerate(cnf.names):
            exp = set(zip(*map(lambda v: v.tolist(), np.nonzero(snaps[it][a]))))
            assert set(map(tuple, qq.get(nm).tolist())) == exp, (it, nm)


# ------------------------------------------------------------------ random graphs and grammars

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("schedule", SCHEDULES)
def test_random_small(seed, schedule):
    graph = synth.random_graph(40 + 7 * seed, 90 + 10 * seed, 3, seed=seed)
    text = synth.random_grammar_text(5, 3, 9, 6, seed % 3, seed=seed)
    assert_parity(graph, text, schedule=schedule)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 255, 256, 257, 300, 513])
def test_ragged_sizes(n):
    graph = synth.random_graph(n, 3 * n, 2, seed=n)
    assert_parity(graph, "S S S\nS A B\nA t0\nB t1\nE eps\nF E S\n")


@pytest.mark.parametrize("seed", range(3))
def test_random_medium_dense(seed):
    # enough closure to make rows dense and span several 256-wide tiles plus a ragged tail
    graph = synth.random_graph(1100, 2600, 2, seed=seed)
    assert_parity(graph, "S S S\nS A B\nS A S1\nS1 S B\nA t0\nB t1\n")


def test_transitive_closure_wide():
    graph = synth.random_graph(3000, 4000, 1, seed=7)
    assert_parity(graph, "S S S\nS t0\n")


def test_empty_and_isolated():
    graph = synth.Graph(n=10, edges=np.zeros((0, 3), dtype=np.int64), labels=["a"])
    g, q, _ = assert_parity(graph, "S S S\nS a\nE eps\n")
    assert q.count("S") == 0 and q.count("E") == 10


def test_duplicate_edges_and_rules():
    graph = synth.random_graph(50, 100, 2, seed=3)
    dup = synth.Graph(n=50, edges=np.concatenate([graph.edges, graph.edges[:40]]), labels=graph.labels)
    assert_parity(dup, "S A B\nS A B\nS S S\nA t0\nA t0\nB t1\n")


def test_no_binary_rules():
    graph = synth.random_graph(20, 30, 2, seed=1)
    g, q, _ = assert_parity(graph, "A t0\nB t1\n")
    assert q.stats()["iterations"] == 1


# ------------------------------------------------------------------ workload shapes

@pytest.mark.parametrize("seed", range(5))
def test_hierarchy_n1024_q1(seed):
    assert_parity(synth.hierarchy(1024, 300, seed=seed), synth.GRAMMAR_Q1)


@pytest.mark.parametrize("text", [synth.GRAMMAR_Q1, synth.GRAMMAR_QSC])
def test_hierarchy_n16384(text):
    assert_parity(synth.hierarchy(16384, 5000, seed=0), text)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_hierarchy_q2_paper(schedule):
    assert_parity(synth.hierarchy(2000, 700, seed=4), synth.GRAMMAR_Q2, schedule=schedule)


@pytest.mark.parametrize("p,q", [(6, 4), (9, 6), (8, 7), (5, 5), (1, 1), (33, 32)])
def test_two_cycles_small(p, q):
    assert_parity(synth.two_cycles(p, q), synth.GRAMMAR_C3)


@pytest.mark.parametrize("p,q", [(2, 1), (3, 2), (5, 4), (9, 8)])
def test_two_cycles_jacobi_iterations(p, q):
    g, qq = solve_engine(synth.two_cycles(p, q), synth.GRAMMAR_C3, schedule=eng.SCHED_JACOBI)
    assert qq.stats()["iterations"] == 2 * p * q + 1


def test_graph_loop_at_depth_two_cycles_64_63():
    """The conditional-while graph of one solve running thousands of loop executions: two
    cycles of 64 and 63 nodes under the Jacobi schedule need k = 2pq + 1 = 8065 executions
    (Lemma 3: derivation height <= k), every one of them launched by the graph (no hand-over
    to the worklist under Jacobi); gcd(64, 63) = 1, so R_S = R_S1 = (a-cycle) x (b-cycle)."""
    p, qn = 64, 63
    graph = synth.two_cycles(p, qn)
    g, q = solve_engine(graph, synth.GRAMMAR_C3, schedule=eng.SCHED_JACOBI, path=eng.PATH_GATHER, use_graph=True)
    s = q.stats()
    assert s["iterations"] == 2 * p * qn + 1 and s["worklist_items"] == 0
    a_nodes = np.arange(p)
    b_nodes = np.concatenate([[0], np.arange(p, p + qn - 1)])
    closed = np.array(sorted((int(i), int(j)) for i in a_nodes for j in b_nodes), dtype=np.uint32)
    assert np.array_equal(q.get("S"), closed)
    ref = oracle.hellings(graph, synth.GRAMMAR_C3)
    for nm in g.names:
        assert np.array_equal(q.get(nm), ref.pairs(nm)), nm


# ------------------------------------------------------------------ limits and statuses

def test_iteration_limit_status_and_partial_result():
    graph = synth.two_cycles(9, 8)
    g = eng.Grammar(synth.GRAMMAR_C3, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, max_iter=5)
    assert q.solve(check=False) == eng.ERR_ITER_LIMIT
    assert q.stats()["iterations"] == 5
    full = oracle.hellings(graph, synth.GRAMMAR_C3).as_sets()
    part = engine_sets(q, g.names)
    for nm in g.names:
        assert part[nm] <= full[nm]


def test_timeout_status():
    # a deadline that has passed before the first iteration ends: the tail reports it
    graph = synth.two_cycles(64, 63)
    g = eng.Grammar(synth.GRAMMAR_C3, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, timeout_s=1e-9)
    assert q.solve(check=False) == eng.ERR_TIMEOUT
    full = oracle.hellings(graph, synth.GRAMMAR_C3).as_sets()
    for nm in g.names:
        assert engine_sets(q, [nm])[nm] <= full[nm]


def test_get_before_solve_and_buffer_too_small():
    graph = synth.random_graph(30, 60, 2, seed=2)
    g = eng.Grammar("S A B\nA t0\nB t1\n", graph.labels)
    q = eng.Query(g, graph.n, graph.edges)
    c = ctypes.c_size_t()
    assert eng.library().cfpq_get(q.handle, 0, None, 0, ctypes.byref(c)) == eng.ERR_NOT_SOLVED
    q.solve()
    k = q.count("S")
    assert k > 0
    buf = (eng.Triple * 1)()
    assert eng.library().cfpq_get(q.handle, 0, buf, 0, ctypes.byref(c)) == eng.ERR_BUFFER
    assert c.value == k


def test_get_device_matches_get():
    import torch
    graph = synth.hierarchy(900, 250, seed=2)
    g, q = solve_engine(graph, synth.GRAMMAR_Q1)
    for nm in g.names:
        k = q.count(nm)
        buf = torch.empty(max(1, k) * 3, dtype=torch.int32, device="cuda")
        assert q.get_device(nm, buf.data_ptr(), max(1, k)) == k
        torch.cuda.synchronize()
        dev = buf[: 3 * k].view(-1, 3).cpu().numpy().astype(np.int64)
        assert np.array_equal(dev, q.triples(nm))


def test_get_all_device_matches_get_all():
    import torch
    graph = synth.hierarchy(900, 250, seed=2)
    g, q = solve_engine(graph, synth.GRAMMAR_Q1)
    k = q.get_all_device(0, 0)
    buf = torch.empty(max(1, k) * 3, dtype=torch.int32, device="cuda")
    assert q.get_all_device(buf.data_ptr(), max(1, k)) == k
    torch.cuda.synchronize()
    dev = buf[: 3 * k].view(-1, 3).cpu().numpy().astype(np.int64)
    assert np.array_equal(dev, q.triples_all())
    with pytest.raises(eng.CfpqError) as ei:
        q.get_all_device(buf.data_ptr(), k - 1)
    assert ei.value.code == eng.ERR_BUFFER


def test_resolve_is_repeatable_and_profile_mode():
    graph = synth.hierarchy(700, 200, seed=9)
    g = eng.Grammar(synth.GRAMMAR_Q1, graph.labels)
    q = eng.Query(g, graph.n, graph.edges)
    q.solve()
    first = engine_sets(q, g.names)
    q.solve()
    assert engine_sets(q, g.names) == first
    qp = eng.Query(g, graph.n, graph.edges, profile=True)
    qp.solve()
    assert engine_sets(qp, g.names) == first
    s = qp.stats()
    # one timed gather unit (scan + listed gathers) per execution, plus each tensor launch
    assert s["product_launches"] == s["iterations"] + s["tensor_launches"] and s["product_ms"] > 0


@pytest.mark.parametrize("text", [synth.GRAMMAR_Q1, synth.GRAMMAR_QSC])
def test_algorithm1_loop_count_matches_oracle(text):
    # the benchmark's work per step is Algorithm 1's loop count x productions: the engine's
    # Jacobi count and the oracle's own sparse Algorithm 1 must agree on it
    graph = synth.hierarchy(16384, 5000, seed=0)
    _, _, k = oracle.matrix_closure_sparse(graph, text)
    for path in (eng.PATH_GATHER, eng.PATH_TENSOR):
        g, q = solve_engine(graph, text, schedule=eng.SCHED_JACOBI, path=path)
        assert q.stats()["iterations"] == k


@pytest.mark.parametrize("n,c", [(700, 200), (5000, 1500)])
def test_get_all_equals_per_relation(n, c):
    graph = synth.hierarchy(n, c, seed=3)
    g, q = solve_engine(graph, synth.GRAMMAR_Q1)
    allt = q.triples_all()
    per = np.concatenate([q.triples(nm) for nm in g.names], axis=0)
    assert np.array_equal(allt, per)


def test_mma_sync_peaks_are_measured():
    p = eng.measure_mma_sync_peaks()
    # both are real device rates: far above zero, far below the FP8 tcgen05 peak (4.5 PF)
    assert 10.0 < p["s8_tops"] < 4500.0 and 10.0 < p["b1_tops"] < 40000.0


def test_serving_workload_large_query_full_size():
    # the served stream's n = 65536 Query 1 query (bit-packed, 7 x 512 MiB per plane set):
    # every relation against the oracle, through the single-query path and through a server
    graph = synth.hierarchy(65536, round(65536 * 0.3), seed=5)
    ref = oracle.hellings(graph, synth.GRAMMAR_Q1)
    g = eng.Grammar(synth.GRAMMAR_Q1, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, timeout_s=300.0)
    q.solve()
    for nm in g.names:
        assert np.array_equal(q.get(nm), ref.pairs(nm)), nm
    q.close()
    srv = eng.Server(rounds_per_step=8)
    t = srv.submit(g, graph.n, graph.edges)
    while srv.stats()["completed"] + srv.stats()["failed"] < 1:
        srv.step()
    assert srv.info(t)["status"] == eng.OK
    for nm in g.names:
        assert np.array_equal(srv.result(t, g.id(nm)), ref.pairs(nm)), nm
    srv.close()


@pytest.mark.parametrize("path,schedule,dense", [
    (eng.PATH_AUTO, eng.SCHED_INPLACE, False), (eng.PATH_GATHER, eng.SCHED_JACOBI, False),
    (eng.PATH_TENSOR, eng.SCHED_INPLACE, False), (eng.PATH_TENSOR, eng.SCHED_JACOBI, True),
    (eng.PATH_WORKLIST, eng.SCHED_INPLACE, False)])
def test_solving_again_starts_from_the_edges(path, schedule, dense):
    # a solve after a converged one clears only the rows of T that hold bits (the delta planes
    # are already zero); after an interrupted one, everything: each solve equals the oracle
    graph = synth.hierarchy(3000, 900, seed=4)
    text = synth.GRAMMAR_Q1
    g = eng.Grammar(text, graph.labels)
    ref = oracle.hellings(graph, text)
    q = eng.Query(g, graph.n, graph.edges, path=path, schedule=schedule, dense_tensor=dense, timeout_s=120.0)
    for _ in range(3):
        q.solve()
        for nm in g.names:
            assert np.array_equal(q.get(nm), ref.pairs(nm)), nm
    if path != eng.PATH_WORKLIST:
        qi = eng.Query(g, graph.n, graph.edges, path=path, schedule=schedule, dense_tensor=dense, max_iter=2)
        assert qi.solve(check=False) == eng.ERR_ITER_LIMIT
        assert qi.solve(check=False) == eng.ERR_ITER_LIMIT
        part = {nm: set(map(tuple, qi.get(nm).tolist())) for nm in g.names}
        full = ref.as_sets()
        assert all(part[nm] <= full[nm] for nm in g.names)


def test_solving_again_after_the_hand_over_to_the_worklist():
    graph = synth.two_cycles(64, 63)
    g = eng.Grammar(synth.GRAMMAR_C3, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_AUTO, timeout_s=120.0)
    ref = oracle.hellings(graph, synth.GRAMMAR_C3)
    for _ in range(2):
        q.solve()
        for nm in g.names:
            assert np.array_equal(q.get(nm), ref.pairs(nm)), nm


@pytest.mark.parametrize("path,schedule", [(eng.PATH_AUTO, eng.SCHED_INPLACE), (eng.PATH_GATHER, eng.SCHED_JACOBI),
                                           (eng.PATH_TENSOR, eng.SCHED_INPLACE), (eng.PATH_WORKLIST, eng.SCHED_INPLACE)])
def test_most_nonterminals(path, schedule):
    # CFPQ_MAX_NONTERM = 64 non-terminals (per-non-terminal arrays, groups and choice threads at
    # their limit); 150 binary productions, 70 unary, 4 with A -> eps
    text = synth.random_grammar_text(64, 3, 150, 70, 4, seed=9)
    graph = synth.random_graph(120, 300, 3, seed=9)
    g = eng.Grammar(text, graph.labels)
    assert len(g.names) == 64
    q = eng.Query(g, graph.n, graph.edges, path=path, schedule=schedule, timeout_s=120.0)
    q.solve()
    ref = oracle.hellings(graph, text)
    for nm in g.names:
        assert np.array_equal(q.get(nm), ref.pairs(nm)), nm


def test_most_nonterminals_batched_and_lengths():
    text = synth.random_grammar_text(64, 3, 150, 70, 4, seed=9)
    graph = synth.random_graph(120, 300, 3, seed=9)
    g = eng.Grammar(text, graph.labels)
    ref = oracle.hellings(graph, text)
    qs = [eng.Query(g, graph.n, graph.edges) for _ in range(3)]
    eng.solve_batch(qs)
    for q in qs:
        for nm in g.names:
            assert np.array_equal(q.get(nm), ref.pairs(nm)), nm
    text_l = synth.random_grammar_text(64, 3, 100, 70, 4, seed=9)
    small = synth.random_graph(40, 60, 3, seed=9)
    gl = eng.Grammar(text_l, small.labels)
    ql = eng.Query(gl, small.n, small.edges, schedule=eng.SCHED_JACOBI, lengths=True, timeout_s=120.0)
    ql.solve()
    cnf, L, _ = oracle.single_path_lengths(small, text_l)
    for a, nm in enumerate(cnf.names):
        pairs, lens = ql.lengths(nm)
        got = {(int(m), int(n)): int(x) for (m, n), x in zip(pairs.tolist(), lens.tolist())}
        assert got == L[a], nm
