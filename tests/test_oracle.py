"""Pins for the CPU oracle: each test checks it against something other than itself.

* the worked example of Section 4.3 (every intermediate matrix T_0..T_5, the loop
  count k = 6 and the relations R_A), read from ``tests/golden/worked_example.txt``;
* brute force over walks with CYK (Section 2's definition of R_A, directly);
* closed forms (two cycles sharing a node; S -> S S | a is transitive closure;
  S -> A B is one Boolean matrix product; the sc-only query on a tree hierarchy);
* Lemma 3 (derivation height <= k after k iterations) on the two-cycle family, where
  the largest minimal height is known in closed form;
* agreement between the worklist oracle and Algorithm 1 written literally;
* planted mistakes: wrong variants of the C oracle must fail these pins.
"""
import math
import os

import numpy as np
import pytest

import cfpq_synth as synth
import oracle


def read_golden(path):
    g = {"edges": [], "T": {}, "R": {}, "k": None, "n": None}
    with open(path) as f:
        for ln in f:
            ln = ln.split("#", 1)[0].strip()
            if not ln:
                continue
            t = ln.split()
            if t[0] == "n":
                g["n"] = int(t[1])
            elif t[0] == "edge":
                g["edges"].append((int(t[1]), t[2], int(t[3])))
            elif t[0] == "k":
                g["k"] = int(t[1])
            elif t[0] == "R":
                g["R"].setdefault(t[1], set()).add((int(t[2]), int(t[3])))
            elif t[0].startswith("T"):
                g["T"].setdefault(int(t[0][1:]), set()).add((int(t[1]), int(t[2]), t[3]))
    return g


@pytest.fixture(scope="module")
def worked(golden_dir):
    return read_golden(os.path.join(golden_dir, "worked_example.txt"))


def test_worked_example_graph_matches_fixture(worked):
    g = synth.worked_example_graph()
    got = sorted((int(s), g.labels[int(l)], int(d)) for s, l, d in g.edges)
    assert got == sorted(worked["edges"])
    assert g.n == worked["n"]


def test_worked_example_relations(worked):
    g = synth.worked_example_graph()
    res = oracle.hellings(g, synth.GRAMMAR_WORKED).as_sets()
    for name in ["S", "S1", "S2", "S3", "S4", "S5", "S6"]:
        assert res[name] == worked["R"].get(name, set()), name


def test_worked_example_every_iteration(worked):
    g = synth.worked_example_graph()
    cnf, snaps, k = oracle.matrix_closure(g, synth.GRAMMAR_WORKED)
    assert k == worked["k"] == 6
    assert len(snaps) == 6  # T_0 .. T_5
    for i, T in enumerate(snaps):
        got = {(int(a), int(b), cnf.names[A]) for A, M in T.items() for a, b in zip(*np.nonzero(M))}
        assert got == worked["T"][i], f"T{i}"


def _as_sets_from_snap(cnf, T):
    return {cnf.names[a]: set(zip(*map(lambda v: v.tolist(), np.nonzero(M)))) for a, M in T.items()}


# ----------------------------------------------------------------------------- brute force

def _dag_graph(n, m, L, seed):
    k = synth.key(seed, 99)
    i = np.arange(m)
    a = synth.uniform_int(k, 3 * i, n)
    b = synth.uniform_int(k, 3 * i + 1, n)
    lab = synth.uniform_int(k, 3 * i + 2, L)
    src, dst = np.minimum(a, b), np.maximum(a, b)
    keep = src < dst
    e = np.stack([src[keep], lab[keep], dst[keep]], axis=1)
    return synth.Graph(n=n, edges=e, labels=[f"t{j}" for j in range(L)])


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_dag_exact(seed):
    # On a DAG every walk has < n edges, so walks up to n-1 edges are all walks.
    n = 5
    g = _dag_graph(n, 9, 2, seed)
    gram = synth.random_grammar_text(n_nt=3, n_terms=2, n_binary=5, n_unary=4,
                                     n_eps=seed % 2, seed=seed)
    res = oracle.hellings(g, gram).as_sets()
    bf = oracle.brute_force(g, gram, max_len=n - 1)
    assert res == bf


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_cyclic_bounded(seed):
    # On cyclic graphs every bounded enumeration is a subset, and a large enough bound
    # reaches the oracle's result exactly.
    g = synth.random_graph(4, 7, 2, seed=seed)
    gram = synth.random_grammar_text(n_nt=3, n_terms=2, n_binary=4, n_unary=3,
                                     n_eps=(seed + 1) % 2, seed=100 + seed)
    res = oracle.hellings(g, gram).as_sets()
    prev = None
    for L in (3, 6, 9):
        bf = oracle.brute_force(g, gram, max_len=L)
        for name in res:
            assert bf[name] <= res[name]
        prev = bf
    assert prev == res


def test_brute_force_worked_example(worked):
    g = synth.worked_example_graph()
    bf = oracle.brute_force(g, synth.GRAMMAR_WORKED, max_len=8)
    for name, pairs in worked["R"].items():
        assert bf[name] == pairs


# ----------------------------------------------------------------------------- closed forms

def _two_cycle_expected(p, q):
    """R_S for S -> a S b | a b on two cycles sharing node 0: (i, j) is in R_S iff some
    m >= 1 has i + m = 0 (mod p) on the a-cycle and m b-steps from 0 reach j, i.e.
    d_i = e_j (mod gcd(p, q)) with d_i = (p - i) mod p and e_j = position of j."""
    g = math.gcd(p, q)
    pos = {0: 0}
    for t in range(q - 1):
        pos[p + t] = t + 1
    out = set()
    for i in range(p):
        d = (p - i) % p
        for j, e in pos.items():
            if (d - e) % g == 0:
                out.add((i, j))
    return out


@pytest.mark.parametrize("p,q", [(6, 4), (9, 6), (8, 7), (5, 5), (3, 2), (1, 1), (4, 1)])
def test_two_cycles_closed_form(p, q):
    g = synth.two_cycles(p, q)
    res = oracle.hellings(g, synth.GRAMMAR_C3)
    exp = _two_cycle_expected(p, q)
    assert set(map(tuple, res.pairs("S").tolist())) == exp
    # S1 -> S B: one b-step after every S pair
    nxt = {int(s): int(d) for s, l, d in g.edges if l == 1}
    assert set(map(tuple, res.pairs("S1").tolist())) == {(i, nxt[j]) for i, j in exp}
    assert res.count("A") == p and res.count("B") == q


@pytest.mark.parametrize("p,q", [(2, 1), (3, 2), (4, 3), (5, 3), (5, 4)])
def test_two_cycles_iteration_count(p, q):
    # Lemma 3: after k loop executions T holds exactly the pairs with a derivation of
    # height <= k. With gcd(p, q) = 1 the largest minimal m with a^m b^m is pq, whose
    # derivation has height 2pq for S and 2pq + 1 for S1 -> S B, so the loop runs
    # 2pq + 1 times before an execution changes nothing.
    g = synth.two_cycles(p, q)
    cnf, snaps, k = oracle.matrix_closure(g, synth.GRAMMAR_C3)
    assert k == 2 * p * q + 1


def _warshall(adj):
    n = adj.shape[0]
    r = adj.copy()
    for k in range(n):
        r = r | (r[:, [k]] & r[[k], :])
    return r


@pytest.mark.parametrize("seed", range(4))
def test_transitive_closure_closed_form(seed):
    g = synth.random_graph(40, 60, 1, seed=seed)
    res = oracle.hellings(g, "S S S\nS t0\n")
    adj = np.zeros((g.n, g.n), dtype=bool)
    adj[g.edges[:, 0], g.edges[:, 2]] = True
    tc = _warshall(adj)
    assert set(map(tuple, res.pairs("S").tolist())) == set(zip(*map(lambda v: v.tolist(), np.nonzero(tc))))


@pytest.mark.parametrize("seed", range(4))
def test_single_product_closed_form(seed):
    g = synth.random_graph(50, 300, 2, seed=seed)
    res = oracle.hellings(g, "S A B\nA t0\nB t1\n")
    A = np.zeros((g.n, g.n), dtype=np.int64)
    B = np.zeros((g.n, g.n), dtype=np.int64)
    for s, l, d in g.edges:
        (A if l == 0 else B)[s, d] = 1
    exp = (A @ B) > 0
    assert set(map(tuple, res.pairs("S").tolist())) == set(zip(*map(lambda v: v.tolist(), np.nonzero(exp))))


@pytest.mark.parametrize("n,C,seed", [(200, 60, 0), (1024, 300, 1), (500, 500, 2)])
def test_sc_only_hierarchy_closed_form(n, C, seed):
    g = synth.hierarchy(n, C, seed=seed)
    res = oracle.hellings(g, synth.GRAMMAR_QSC)
    parent = {int(s): int(d) for s, l, d in g.edges if l == 0}
    has_child = set(parent.values())
    assert set(map(tuple, res.pairs("S").tolist())) == {(p, p) for p in has_child}
    assert set(map(tuple, res.pairs("X").tolist())) == {(c, parent[c]) for c in has_child if c in parent}


def class_depths(g):
    """Depth of every class below the root (class 0) from the generator's sc edges."""
    parent = {int(s): int(d) for s, l, d in g.edges if l == 0}
    C = g.meta["n_classes"]
    depth = [0] * C
    for c in range(1, C):  # parents are earlier classes
        depth[c] = depth[parent[c]] + 1
    return parent, depth


@pytest.mark.parametrize("n,C,seed", [(200, 60, 0), (1024, 300, 1), (2000, 700, 3)])
def test_same_generation_hierarchy_closed_form(n, C, seed):
    # S -> sc S sc_r | sc sc_r: up k >= 1 subClassOf edges then down k. On a tree every two
    # classes at the same depth d >= 1 meet at the root after d steps up, and nothing else
    # qualifies (instances have no sc edges); X = S sc_r adds one step down
    g = synth.hierarchy(n, C, seed=seed)
    res = oracle.hellings(g, synth.GRAMMAR_SG)
    parent, depth = class_depths(g)
    by_depth = {}
    for c, d in enumerate(depth):
        by_depth.setdefault(d, []).append(c)
    exp_s = {(x, y) for d, cs in by_depth.items() if d >= 1 for x in cs for y in cs}
    assert set(map(tuple, res.pairs("S").tolist())) == exp_s
    exp_x = {(x, c) for (x, y) in exp_s for c in by_depth.get(depth[y] + 1, []) if parent.get(c) == y}
    assert set(map(tuple, res.pairs("X").tolist())) == exp_x


def test_q1_hierarchy_y_empty():
    g = synth.hierarchy(1024, 300, seed=0)
    res = oracle.hellings(g, synth.GRAMMAR_Q1)
    assert res.count("Y") == 0
    assert res.count("S") > 0


# ----------------------------------------------------------------------------- cross-checks

@pytest.mark.parametrize("seed", range(6))
def test_worklist_equals_algorithm1(seed):
    g = synth.random_graph(24, 60, 3, seed=seed)
    gram = synth.random_grammar_text(n_nt=5, n_terms=3, n_binary=9, n_unary=6,
                                     n_eps=seed % 3, seed=seed)
    res = oracle.hellings(g, gram).as_sets()
    cnf, snaps, k = oracle.matrix_closure(g, gram)
    final = _as_sets_from_snap(cnf, snaps[-1])
    assert res == final


@pytest.mark.parametrize("seed", range(3))
def test_monotone_iterations(seed):
    g = synth.random_graph(20, 50, 2, seed=seed)
    gram = synth.random_grammar_text(4, 2, 7, 4, 0, seed=seed)
    cnf, snaps, k = oracle.matrix_closure(g, gram)
    for a, b in zip(snaps, snaps[1:]):
        for A in a:
            assert (b[A] >= a[A]).all()  # a^(i) contains a^(i-1)
    # Theorem 3: at most |V|^2 |N| changing iterations
    assert k - 1 <= g.n * g.n * len(cnf.names)


@pytest.mark.parametrize("seed", range(3))
def test_properties_hold_on_oracle(seed):
    g = synth.hierarchy(300, 90, seed=seed)
    cnf = oracle.parse_grammar(synth.GRAMMAR_Q1, g.labels)
    res = oracle.hellings(g, synth.GRAMMAR_Q1)
    sets = {nm: res.pairs(nm) for nm in cnf.names}
    assert oracle.check_seed_included(cnf, g.n, g.edges, sets)
    assert oracle.check_closed(cnf, g.n, sets)
    assert oracle.check_witnessed(cnf, g.n, g.edges, sets)


# ----------------------------------------------------------------------------- grammar reader

def test_grammar_reader_q1_normal_form():
    cnf = oracle.parse_grammar(synth.GRAMMAR_Q1, synth.HIERARCHY_LABELS)
    assert cnf.names == ["S", "X", "Y", "SC", "TY", "<sc_r>", "<ty_r>"]
    assert len(cnf.binary) == 6 and len(cnf.unary) == 4 and cnf.eps == []


def test_grammar_reader_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.parse_grammar("S A\nA a\n", ["a"])        # chain rule
    with pytest.raises(ValueError):
        oracle.parse_grammar("S zz\n", ["a"])            # unknown terminal
    with pytest.raises(ValueError):
        oracle.parse_grammar("S a b c\n", ["a", "b", "c"])


def test_oracle_rejects_out_of_range_edges():
    g = synth.Graph(n=3, edges=np.array([[0, 0, 5]]), labels=["a"])
    with pytest.raises(ValueError):
        oracle.hellings(g, "S a\n")


def test_empty_graph_and_isolated_nodes():
    g = synth.Graph(n=4, edges=np.zeros((0, 3), dtype=np.int64), labels=["a"])
    res = oracle.hellings(g, "S S S\nS a\nE eps\n")
    assert res.count("S") == 0
    assert set(map(tuple, res.pairs("E").tolist())) == {(i, i) for i in range(4)}


# ----------------------------------------------------------------------------- planted mistakes

@pytest.mark.parametrize("plant", [1, 2, 3])
def test_planted_mistakes_are_caught(plant, worked):
    """Each deliberately wrong build of the C oracle must fail at least one pin."""
    failures = 0
    g = synth.worked_example_graph()
    res = oracle.hellings(g, synth.GRAMMAR_WORKED, plant=plant).as_sets()
    failures += any(res[nm] != worked["R"].get(nm, set()) for nm in res)
    for seed in range(4):
        gg = synth.random_graph(4, 7, 2, seed=seed)
        gram = synth.random_grammar_text(3, 2, 4, 3, 1, seed=100 + seed)
        r = oracle.hellings(gg, gram, plant=plant).as_sets()
        failures += r != oracle.brute_force(gg, gram, max_len=9)
    assert failures > 0


# ----------------------------------------------------------------------------- sparse Algorithm 1

def test_sparse_algorithm1_worked_example(worked):
    cnf, T, k = oracle.matrix_closure_sparse(synth.worked_example_graph(), synth.GRAMMAR_WORKED)
    assert k == worked["k"] == 6
    for a, nm in enumerate(cnf.names):
        coo = T[a].tocoo()
        assert set(zip(coo.row.tolist(), coo.col.tolist())) == worked["R"].get(nm, set())


@pytest.mark.parametrize("p,q", [(3, 2), (5, 4), (7, 3)])
def test_sparse_algorithm1_two_cycle_count(p, q):
    _, _, k = oracle.matrix_closure_sparse(synth.two_cycles(p, q), synth.GRAMMAR_C3)
    assert k == 2 * p * q + 1


@pytest.mark.parametrize("seed", range(4))
def test_sparse_algorithm1_equals_dense(seed):
    g = synth.random_graph(30, 70, 3, seed=seed)
    gram = synth.random_grammar_text(5, 3, 9, 6, seed % 2, seed=seed)
    cnf, snaps, k = oracle.matrix_closure(g, gram)
    cnf2, T, k2 = oracle.matrix_closure_sparse(g, gram)
    assert k == k2
    for a in range(len(cnf.names)):
        assert (T[a].toarray() != 0).tolist() == snaps[-1][a].tolist()


def test_property_checks_detect_broken_results():
    """The property checks must reject results with a pair removed or a seed missing."""
    g = synth.hierarchy(300, 90, seed=7)
    cnf = oracle.parse_grammar(synth.GRAMMAR_Q1, g.labels)
    res = oracle.hellings(g, synth.GRAMMAR_Q1)
    good = {nm: res.pairs(nm) for nm in cnf.names}
    assert oracle.check_closed(cnf, g.n, good) and oracle.check_seed_included(cnf, g.n, g.edges, good)
    # drop a derived pair of S: the closure check fails (some product now points outside R_S)
    broken = dict(good)
    x_pairs = good["X"]
    # an S pair that is produced from SCR x X: remove it
    scr = set(map(tuple, good["<sc_r>"].tolist()))
    xs = set(map(tuple, x_pairs.tolist()))
    produced = {(i, j) for (i, k) in scr for (k2, j) in xs if k == k2}
    victim = sorted(produced)[0]
    broken["S"] = np.array([p for p in good["S"].tolist() if tuple(p) != victim], dtype=np.uint32)
    assert not oracle.check_closed(cnf, g.n, broken)
    # drop a seed pair
    broken2 = dict(good)
    broken2["SC"] = good["SC"][1:]
    assert not oracle.check_seed_included(cnf, g.n, g.edges, broken2)
    # add a pair with no derivation: the witness check fails
    broken3 = dict(good)
    broken3["S"] = np.concatenate([good["S"], np.array([[g.n - 1, g.n - 1]], dtype=np.uint32)])
    assert not oracle.check_witnessed(cnf, g.n, g.edges, broken3)


# ----------------------------------------------------------------------------- single-path lengths (Section 5)

def _labelled(n, edges, labels):
    return synth.Graph(n=n, edges=np.asarray(edges, dtype=np.int64).reshape(-1, 3), labels=list(labels),
                       meta={"kind": "test"})


@pytest.mark.parametrize("n", [2, 9, 40])
def test_lengths_on_a_path_are_distances(n):
    # S -> S S | a on a directed path: the only walk from i to j has j - i edges
    g = _labelled(n, [(i, 0, i + 1) for i in range(n - 1)], ["a"])
    cnf, L, k = oracle.single_path_lengths(g, "S S S\nS a\n")
    assert len(L[0]) == n * (n - 1) // 2
    assert all(l == j - i for (i, j), l in L[0].items())


@pytest.mark.parametrize("p,q", [(5, 4), (7, 3), (6, 5), (3, 2), (1, 1)])
def test_lengths_on_two_cycles_closed_form(p, q):
    # S -> a S b | a b: a walk a^k b^k from a-node i must pass node 0 after k a-steps, so
    # k = d_i (mod p) and k = e_j (mod q); derivations of smaller k appear in earlier loop
    # executions, so the length found first is 2 k_min
    g = synth.two_cycles(p, q)
    cnf, L, k = oracle.single_path_lengths(g, synth.GRAMMAR_C3)
    S = cnf.names.index("S")
    bnodes = [0] + list(range(p, p + q - 1))
    assert len(L[S]) == p * q  # gcd(p, q) = 1: every (a-node, b-node) pair
    for (i, j), l in L[S].items():
        d, e = (p - i) % p, bnodes.index(j)
        kmin = next(kk for kk in range(1, 2 * p * q + 2) if kk % p == d % p and kk % q == e % q)
        assert l == 2 * kmin, (i, j)


@pytest.mark.parametrize("seed", range(5))
def test_lengths_have_witness_walks(seed):
    # Theorem 5 of Section 5: (A, l) at (i, j) means a walk of exactly l edges from i to j
    # whose labels A derives (brute force: every walk of that length, CYK on its labels)
    g = synth.random_graph(6, 9, 2, seed=seed)
    text = synth.random_grammar_text(4, 2, 6, 4, seed % 2, seed=seed)
    cnf, L, k = oracle.single_path_lengths(g, text, max_iter=6)
    for a, pairs in L.items():
        for (i, j), l in pairs.items():
            if l <= 7:
                assert oracle.walk_exists(g, cnf, a, i, j, l), (cnf.names[a], i, j, l)


@pytest.mark.parametrize("seed", range(4))
def test_lengths_cover_the_relational_result(seed):
    # the pairs carrying a length are exactly R_A (the relational result)
    g = synth.random_graph(30, 70, 3, seed=seed)
    text = synth.random_grammar_text(5, 3, 9, 6, seed % 3, seed=seed)
    cnf, L, k = oracle.single_path_lengths(g, text)
    ref = oracle.hellings(g, text).as_sets()
    for a, name in enumerate(cnf.names):
        assert set(L[a]) == ref[name]
    # and the loop runs exactly as many executions as Algorithm 1
    assert k == oracle.matrix_closure(g, text)[2]


def _diamond():
    # two walks from 0 to 3: 0-1-2-3 (3 edges) and 0-4-5-6-3 (4 edges); with S -> S S | a both
    # complete in the same loop execution (lengths in (2, 4]), and the smaller is kept
    return _labelled(7, [(0, 0, 1), (1, 0, 2), (2, 0, 3), (0, 0, 4), (4, 0, 5), (5, 0, 6), (6, 0, 3)], ["a"])


def test_lengths_tie_in_one_execution_keeps_the_smallest():
    cnf, L, _ = oracle.single_path_lengths(_diamond(), "S S S\nS a\n")
    assert L[0][(0, 3)] == 3


@pytest.mark.parametrize("plant", ["plus_one", "last_wins", "max_tie"])
def test_lengths_planted_mistakes_fail_a_pin(plant):
    # each run is capped well above the executions Algorithm 1 needs there, and "the loop ends
    # before the cap" is a pin of its own (a length that keeps changing never lets it end)
    cap = 40
    failed = []
    path = _labelled(12, [(i, 0, i + 1) for i in range(11)], ["a"])
    _, L, k = oracle.single_path_lengths(path, "S S S\nS a\n", max_iter=cap, _plant=plant)
    failed.append(k >= cap or any(l != j - i for (i, j), l in L[0].items()))
    _, L, k = oracle.single_path_lengths(_diamond(), "S S S\nS a\n", max_iter=cap, _plant=plant)
    failed.append(k >= cap or L[0][(0, 3)] != 3)
    p, q = 3, 2
    g = synth.two_cycles(p, q)
    cnf, L, k = oracle.single_path_lengths(g, synth.GRAMMAR_C3, max_iter=cap, _plant=plant)
    S = cnf.names.index("S")
    bnodes = [0] + list(range(p, p + q - 1))
    wrong = k >= cap
    for (i, j), l in L[S].items():
        d, e = (p - i) % p, bnodes.index(j)
        kmin = next(kk for kk in range(1, 2 * p * q + 2) if kk % p == d % p and kk % q == e % q)
        wrong |= l != 2 * kmin
    failed.append(wrong)
    assert any(failed), plant
