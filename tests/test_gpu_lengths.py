"""Single-path semantics (Section 5) on the device: every pair of R_A carries the length of one
walk, set by the loop execution that first derives the pair (smallest of that execution's
derivations). Compared pair by pair and length by length with the oracle, on every matrix
path, and at full size through properties that hold at any size."""
import ctypes

import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu

PATHS = [eng.PATH_GATHER, eng.PATH_TENSOR, eng.PATH_AUTO]


def solve_lengths(graph, text, path=eng.PATH_AUTO, schedule=eng.SCHED_JACOBI, **kw):
    kw.setdefault("timeout_s", 300.0)
    g = eng.Grammar(text, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=path, schedule=schedule, lengths=True, **kw)
    q.solve()
    return g, q


def as_dict(q, name):
    pairs, lens = q.lengths(name)
    return {(int(m), int(n)): int(l) for (m, n), l in zip(pairs.tolist(), lens.tolist())}


def parity(graph, text, path=eng.PATH_AUTO, **kw):
    g, q = solve_lengths(graph, text, path=path, **kw)
    cnf, L, k = oracle.single_path_lengths(graph, text)
    assert g.names == cnf.names
    for a, nm in enumerate(cnf.names):
        got = as_dict(q, nm)
        assert set(got) == set(L[a]), nm
        bad = [(p, got[p], L[a][p]) for p in L[a] if got[p] != L[a][p]]
        assert not bad, (nm, bad[:5])
    assert q.stats()["iterations"] == k  # the same loop as Algorithm 1 under the Jacobi schedule
    return g, q


@pytest.mark.parametrize("path", PATHS)
def test_worked_example(path):
    parity(synth.worked_example_graph(), synth.GRAMMAR_WORKED, path)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("seed", range(5))
def test_random(path, seed):
    graph = synth.random_graph(40 + 13 * seed, 100 + 25 * seed, 3, seed=seed)
    parity(graph, synth.random_grammar_text(5, 3, 9, 6, seed % 3, seed=seed), path)


@pytest.mark.parametrize("n", [1, 31, 33, 257, 600])
def test_ragged_sizes_with_eps(n):
    # A -> eps (length 0 on the diagonal) next to loop edges of the same non-terminal
    e = synth.random_graph(n, 3 * n, 2, seed=n).edges
    e = np.concatenate([e, np.array([[m, 0, m] for m in range(0, n, 5)], dtype=np.int64).reshape(-1, 3)])
    graph = synth.Graph(n=n, edges=e, labels=["t0", "t1"], meta={"kind": "test"})
    parity(graph, "S S S\nS A B\nA t0\nA eps\nB t1\nE eps\nF E S\n")


@pytest.mark.parametrize("text", [synth.GRAMMAR_Q1, synth.GRAMMAR_QSC, synth.GRAMMAR_Q2, synth.GRAMMAR_SG])
def test_hierarchy(text):
    parity(synth.hierarchy(3000, 900, seed=6), text)


def test_schedule_auto_is_taken_as_jacobi():
    graph = synth.hierarchy(1000, 300, seed=2)
    g, q = parity(graph, synth.GRAMMAR_Q1, schedule=eng.SCHED_AUTO)
    assert q.stats()["schedule"] == eng.SCHED_JACOBI


def test_tie_in_one_execution_keeps_the_smallest():
    # 0-1-2-3 (3 edges) and 0-4-5-6-3 (4 edges): S -> S S | a derives (0, 3) both ways in the
    # same loop execution; the smaller length is kept
    e = [(0, 0, 1), (1, 0, 2), (2, 0, 3), (0, 0, 4), (4, 0, 5), (5, 0, 6), (6, 0, 3)]
    graph = synth.Graph(n=7, edges=np.array(e, dtype=np.int64), labels=["a"], meta={"kind": "test"})
    for path in PATHS:
        g, q = solve_lengths(graph, "S S S\nS a\n", path)
        assert as_dict(q, "S")[(0, 3)] == 3


@pytest.mark.parametrize("n", [1000, 8192])
def test_path_lengths_are_distances(n):
    # the only walk from i to j on a directed path has j - i edges: n (n - 1) / 2 pairs
    graph = synth.Graph(n=n, edges=np.array([(i, 0, i + 1) for i in range(n - 1)], dtype=np.int64),
                        labels=["a"], meta={"kind": "test"})
    g, q = solve_lengths(graph, "S S S\nS a\n")
    pairs, lens = q.lengths("S")
    assert pairs.shape[0] == n * (n - 1) // 2
    assert np.array_equal(lens.astype(np.int64), pairs[:, 1].astype(np.int64) - pairs[:, 0])


@pytest.mark.parametrize("p,qq", [(9, 8), (33, 32), (128, 127)])
def test_two_cycles_closed_form(p, qq):
    # S -> a S b | a b: the pair (i, j) first appears through a^k b^k with the smallest k such
    # that k = d_i (mod p) and k = e_j (mod q) (d_i, e_j the steps to and from node 0)
    graph = synth.two_cycles(p, qq)
    g, q = solve_lengths(graph, synth.GRAMMAR_C3)
    pairs, lens = q.lengths("S")
    assert pairs.shape[0] == p * qq
    i = pairs[:, 0].astype(np.int64)
    j = pairs[:, 1].astype(np.int64)
    d = (p - i) % p
    e = np.where(j == 0, 0, j - p + 1)
    # CRT by search over one period of the a-cycle: k = d + p t, t = 0 .. q - 1
    t = np.arange(qq, dtype=np.int64)
    ks = d[:, None] + p * t[None, :]
    ks = np.where(ks == 0, p * qq, ks)  # k >= 1: the pair (0, 0) closes after p q steps
    ok = (ks % qq) == (e[:, None] % qq)
    kmin = np.where(ok, ks, np.iinfo(np.int64).max).min(axis=1)
    assert np.array_equal(lens.astype(np.int64), 2 * kmin)
    if p <= 33:
        parity(graph, synth.GRAMMAR_C3)


def _sorted_lookup(pairs, lens, n):
    key = pairs[:, 0].astype(np.int64) * n + pairs[:, 1].astype(np.int64)
    order = np.argsort(key)
    return key[order], lens[order].astype(np.int64)


def _witness_check(graph, text, q, sample, seed):
    """Every length is a seed length (1 for an edge, 0 for A -> eps on the diagonal) or the sum
    l_B(i, k) + l_C(k, j) over some production A -> B C and middle node k of the final
    relations (a length, once set, never changes, so its witness split stays)."""
    cnf = oracle.parse_grammar(text, graph.labels)
    n = graph.n
    tabs = {}
    for a, nm in enumerate(cnf.names):
        pairs, lens = q.lengths(nm)
        tabs[a] = (pairs, lens, *_sorted_lookup(pairs, lens, n))
    seed_len = {}
    heads = {}
    for a, t in cnf.unary:
        heads.setdefault(t, []).append(a)
    for s_, lab, d_ in np.asarray(graph.edges).reshape(-1, 3).tolist():
        for a in heads.get(lab, []):
            seed_len[(a, s_, d_)] = 1
    for a in cnf.eps:
        for m in range(n):
            seed_len[(a, m, m)] = 0
    rng = np.random.default_rng(seed)
    checked = 0
    for a in range(len(cnf.names)):
        pairs, lens, keys, lsorted = tabs[a]
        if pairs.shape[0] == 0:
            continue
        idx = rng.choice(pairs.shape[0], size=min(sample, pairs.shape[0]), replace=False)
        for t in idx.tolist():
            i, j, l = int(pairs[t, 0]), int(pairs[t, 1]), int(lens[t])
            if (a, i, j) in seed_len:
                assert l == seed_len[(a, i, j)], (cnf.names[a], i, j, l)
                continue
            found = False
            for (lhs, b, c) in cnf.binary:
                if lhs != a or found:
                    continue
                _, _, kb, lb_sorted = tabs[b]
                _, _, kc, lc_sorted = tabs[c]
                lo, hi = np.searchsorted(kb, [i * n, (i + 1) * n])
                if hi == lo or len(kc) == 0:
                    continue
                want = (kb[lo:hi] - i * n) * n + j  # (k, j) for every k with (i, k) in R_B
                pos = np.minimum(np.searchsorted(kc, want), len(kc) - 1)
                hit = kc[pos] == want
                found = bool(np.any(hit & (lb_sorted[lo:hi] + lc_sorted[pos] == l)))
            assert found, (cnf.names[a], i, j, l)
            checked += 1
    return checked


def test_full_size_hierarchy_parity():
    """The benchmark's same-generation query at n = 16384 (5000 classes), every pair and
    length against the oracle (about 7 s on the host)."""
    graph = synth.hierarchy(16384, 5000, seed=1)
    parity(graph, synth.GRAMMAR_Q1)


@pytest.mark.parametrize("text", [synth.GRAMMAR_SG, synth.GRAMMAR_Q2])
def test_full_size_hierarchy_witnesses(text):
    graph = synth.hierarchy(16384, 5000, seed=1)
    g, q = solve_lengths(graph, text)
    ref = oracle.matrix_closure_sparse(graph, text)
    cnf, T, k = ref
    for a, nm in enumerate(cnf.names):
        assert q.count(nm) == T[a].nnz, nm
    assert q.stats()["iterations"] == k
    assert _witness_check(graph, text, q, 300, seed=7) > 0


def test_profile_counts_the_length_launches():
    graph = synth.hierarchy(3000, 900, seed=6)
    g, q = solve_lengths(graph, synth.GRAMMAR_Q1, profile=True)
    st = q.stats()
    assert st["lengths_launches"] == st["iterations"] and st["lengths_ms"] > 0
    assert st["lengths_splits"] >= st["new_bits"]  # every new pair has at least one split
    parity(graph, synth.GRAMMAR_Q1, profile=True, use_graph=False)


def test_repeated_solve_gives_the_same_lengths():
    graph = synth.random_graph(300, 900, 3, seed=4)
    text = synth.random_grammar_text(5, 3, 9, 6, 1, seed=4)
    g, q = solve_lengths(graph, text)
    first = {nm: as_dict(q, nm) for nm in g.names}
    q.solve()
    assert {nm: as_dict(q, nm) for nm in g.names} == first


def test_lengths_unavailable_without_the_option_and_in_batches():
    graph = synth.random_graph(50, 120, 3, seed=1)
    text = synth.random_grammar_text(5, 3, 9, 6, 0, seed=1)
    g = eng.Grammar(text, graph.labels)
    plain = eng.Query(g, graph.n, graph.edges)
    plain.solve()
    c = ctypes.c_size_t()
    assert eng.library().cfpq_get_lengths(plain.handle, 0, None, None, 0, ctypes.byref(c)) == eng.ERR_UNSUPPORTED
    _, withlen = solve_lengths(graph, text)
    with pytest.raises(eng.CfpqError) as ei:
        eng.solve_batch([withlen])
    assert ei.value.code == eng.ERR_UNSUPPORTED


# ----------------------------------------------------------------------------- walks (Section 5)

_EDGE_SETS = {}


def _edge_set(graph):
    key = id(graph)
    if key not in _EDGE_SETS:
        _EDGE_SETS.clear()
        _EDGE_SETS[key] = (graph, set(map(tuple, np.asarray(graph.edges).reshape(-1, 3).tolist())))
    return _EDGE_SETS[key][1]


def _check_walk(graph, cnf, a, m, n, length, nodes, labels, cyk_up_to=24):
    """The walk starts at m, ends at n, has the reported length, uses only edges of the graph
    and (for short walks) its label string is derived from A (CYK)."""
    assert len(labels) == length and len(nodes) == length + 1
    assert int(nodes[0]) == m and int(nodes[-1]) == n
    edges = _edge_set(graph)
    for t in range(length):
        assert (int(nodes[t]), int(labels[t]), int(nodes[t + 1])) in edges, (t, nodes[t], labels[t], nodes[t + 1])
    if length <= cyk_up_to:
        assert a in oracle.cyk_table(cnf, [int(x) for x in labels])[0][length]


@pytest.mark.parametrize("seed", range(4))
def test_every_pair_has_a_walk_of_its_length(seed):
    graph = synth.random_graph(30 + 7 * seed, 70 + 15 * seed, 3, seed=seed)
    text = synth.random_grammar_text(5, 3, 9, 6, seed % 3, seed=seed)
    g, q = solve_lengths(graph, text)
    cnf = oracle.parse_grammar(text, graph.labels)
    checked = 0
    for a, nm in enumerate(cnf.names):
        pairs, lens = q.lengths(nm)
        for (m, n), l in zip(pairs.tolist()[:60], lens.tolist()[:60]):
            nodes, labels = q.path(nm, m, n)
            _check_walk(graph, cnf, a, m, n, l, nodes, labels)
            checked += 1
    assert checked > 0


def test_walks_on_two_cycles_are_a_k_b_k():
    p, qq = 33, 32
    graph = synth.two_cycles(p, qq)
    g, q = solve_lengths(graph, synth.GRAMMAR_C3)
    cnf = oracle.parse_grammar(synth.GRAMMAR_C3, graph.labels)
    pairs, lens = q.lengths("S")
    for (m, n), l in list(zip(pairs.tolist(), lens.tolist()))[::37]:
        nodes, labels = q.path("S", m, n)
        k = l // 2
        assert labels.tolist() == [0] * k + [1] * k
        _check_walk(graph, cnf, cnf.names.index("S"), m, n, l, nodes, labels)


def test_empty_walk_missing_pair_and_determinism():
    graph = synth.Graph(n=4, edges=np.array([(0, 0, 1), (1, 1, 2), (0, 0, 1)], dtype=np.int64),
                        labels=["t0", "t1"], meta={"kind": "test"})
    text = "S A B\nA t0\nB t1\nE eps\n"
    g, q = solve_lengths(graph, text)
    nodes, labels = q.path("E", 3, 3)
    assert nodes.tolist() == [3] and labels.size == 0
    nodes, labels = q.path("S", 0, 2)
    assert nodes.tolist() == [0, 1, 2] and labels.tolist() == [0, 1]
    with pytest.raises(eng.CfpqError) as ei:
        q.path("S", 2, 0)
    assert ei.value.code == eng.ERR_NOT_FOUND
    c = ctypes.c_size_t()
    small = (ctypes.c_uint32 * 2)()
    lab = (ctypes.c_int32 * 1)()
    assert eng.library().cfpq_get_path(q.handle, g.id("S"), 0, 2, small, lab, 1, ctypes.byref(c)) == eng.ERR_BUFFER
    assert c.value == 2
    graph2 = synth.hierarchy(2000, 600, seed=3)
    g2, q2 = solve_lengths(graph2, synth.GRAMMAR_SG)
    pairs, _ = q2.lengths("S")
    for m, n in pairs.tolist()[::997]:
        a1, b1 = q2.path("S", m, n)
        a2, b2 = q2.path("S", m, n)
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2)


@pytest.mark.parametrize("text", [synth.GRAMMAR_Q1, synth.GRAMMAR_SG])
def test_full_size_hierarchy_walks(text):
    graph = synth.hierarchy(16384, 5000, seed=1)
    g, q = solve_lengths(graph, text)
    cnf = oracle.parse_grammar(text, graph.labels)
    rng = np.random.default_rng(3)
    for a, nm in enumerate(cnf.names):
        pairs, lens = q.lengths(nm)
        if pairs.shape[0] == 0:
            continue
        for t in rng.choice(pairs.shape[0], size=min(40, pairs.shape[0]), replace=False).tolist():
            m, n, l = int(pairs[t, 0]), int(pairs[t, 1]), int(lens[t])
            nodes, labels = q.path(nm, m, n)
            _check_walk(graph, cnf, a, m, n, l, nodes, labels, cyk_up_to=16)


@pytest.mark.parametrize("path", [eng.PATH_GATHER, eng.PATH_AUTO])
def test_graph_solve_runs_the_lengths_in_the_persistent_loop(path):
    """Gather-only executions of a graph solve run in one persistent loop launch that also
    computes the new pairs' lengths (between the gathers and the merge); the host-driven loop
    launches the length kernel once per execution. Same lengths as the oracle either way, and
    the graph solve runs far fewer kernels."""
    graph = synth.hierarchy(2000, 600, seed=4)
    _, qg = parity(graph, synth.GRAMMAR_Q1, path)
    _, qh = parity(graph, synth.GRAMMAR_Q1, path, use_graph=False)
    sg, sh = qg.stats(), qh.stats()
    assert sg["iterations"] == sh["iterations"] > 4
    assert sg["kernel_launches"] < sh["kernel_launches"] - 2 * sh["iterations"]
    qg.close()
    qh.close()
