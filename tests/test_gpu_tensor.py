"""Tensor-core (tcgen05) product path against the CPU oracle, bit-exact."""
import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu

# operand formats of the tensor products: E4M3 bytes (kind::f8f6f4), E2M1 nibbles (kind::mxf4)
KINDS = pytest.mark.parametrize("kind", [eng.TENSOR_FP8, eng.TENSOR_FP4], ids=["fp8", "fp4"])


def tensor_parity(graph, text, **kw):
    kw.setdefault("timeout_s", 120.0)
    g = eng.Grammar(text, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_TENSOR, **kw)
    q.solve()
    ref = oracle.hellings(graph, text)
    for nm in g.names:
        got, exp = q.get(nm), ref.pairs(nm)
        assert got.shape == exp.shape and np.array_equal(got, exp), \
            f"{nm}: engine {got.shape[0]} pairs, oracle {exp.shape[0]}"
    s = q.stats()
    assert s["tensor_products"] > 0 or s["iterations"] <= 1
    return g, q


@KINDS
@pytest.mark.parametrize("n,m", [(200, 3000), (256, 20000), (700, 30000)])
def test_single_product(n, m, kind):
    # S -> A B is one Boolean matrix product: exercises the GEMM, its K loop and epilogue
    tensor_parity(synth.random_graph(n, m, 2, seed=n), "S A B\nA t0\nB t1\n", tensor_kind=kind)


def test_worked_example():
    tensor_parity(synth.worked_example_graph(), synth.GRAMMAR_WORKED)


def test_worked_example_jacobi_iterations():
    g, q = tensor_parity(synth.worked_example_graph(), synth.GRAMMAR_WORKED, schedule=eng.SCHED_JACOBI)
    assert q.stats()["iterations"] == 6


@KINDS
@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("schedule", [eng.SCHED_INPLACE, eng.SCHED_JACOBI])
@pytest.mark.parametrize("dense", [False, True])
def test_random(seed, schedule, dense, kind):
    graph = synth.random_graph(90 + 61 * seed, 200 + 40 * seed, 3, seed=seed)
    text = synth.random_grammar_text(5, 3, 9, 6, seed % 3, seed=seed)
    tensor_parity(graph, text, schedule=schedule, dense_tensor=dense, tensor_kind=kind)


@KINDS
@pytest.mark.parametrize("n", [1100, 2600])
def test_dense_closure(n, kind):
    tensor_parity(synth.random_graph(n, int(1.6 * n), 1, seed=n), "S S S\nS t0\n", tensor_kind=kind)


def test_two_cycles():
    tensor_parity(synth.two_cycles(17, 12), synth.GRAMMAR_C3)


@KINDS
@pytest.mark.parametrize("n,c", [(1024, 300), (4096, 1200)])
@pytest.mark.parametrize("dense", [False, True])
def test_hierarchy_q1(n, c, dense, kind):
    g, q = tensor_parity(synth.hierarchy(n, c, seed=1), synth.GRAMMAR_Q1, dense_tensor=dense, tensor_kind=kind)
    s = q.stats()
    if dense:
        assert s["tensor_live_ops"] == s["dense_ops"]
    else:  # classes and instances occupy separate index ranges: most operand tiles are zero
        assert 0 < s["tensor_live_ops"] < 0.5 * s["dense_ops"]


@KINDS
@pytest.mark.parametrize("text", [synth.GRAMMAR_Q1, synth.GRAMMAR_QSC])
def test_hierarchy_n16384(text, kind):
    tensor_parity(synth.hierarchy(16384, 5000, seed=0), text, tensor_kind=kind)


def test_useful_work_of_one_product():
    # S -> A B, A -> t0, B -> t1: every execution multiplies the same seeded A and B, whose
    # useful multiply-adds are sum_k (ones in column k of A) (ones in row k of B)
    graph = synth.random_graph(700, 9000, 2, seed=11)
    text = "S A B\nA t0\nB t1\n"
    g = eng.Grammar(text, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_TENSOR, schedule=eng.SCHED_JACOBI, profile=True)
    q.solve()
    e = np.unique(np.asarray(graph.edges, dtype=np.int64), axis=0)
    a = e[e[:, 1] == 0]
    b = e[e[:, 1] == 1]
    col_a = np.bincount(a[:, 2], minlength=graph.n)
    row_b = np.bincount(b[:, 0], minlength=graph.n)
    s = q.stats()
    assert s["useful_ops"] == 2.0 * s["iterations"] * float(np.dot(col_a, row_b))
    assert 0 < s["useful_ops"] < s["dense_ops"]


def _block_edges(n, m, label, src_range, dst_range, seed):
    k = synth.key(seed, 5)
    i = np.arange(m, dtype=np.int64)
    src = src_range[0] + synth.uniform_int(k, 2 * i, src_range[1] - src_range[0])
    dst = dst_range[0] + synth.uniform_int(k, 2 * i + 1, dst_range[1] - dst_range[0])
    return np.stack([src, np.full_like(src, label), dst], axis=1)


@KINDS
@pytest.mark.parametrize("schedule", [eng.SCHED_JACOBI, eng.SCHED_INPLACE])
def test_tile_skipping_issues_exactly_the_live_steps(schedule, kind):
    """S -> A B with A and B static: every execution multiplies the same operands, so the K
    steps issued are (executions) x sum over output tiles (128 x 256) of the K steps in which
    A's tile and B^T's tile are both non-zero, counted here from the edge list. An FP8 step is
    one K slice of 128; an FP4 step two consecutive slices, live if either slice is."""
    n = 1024
    e = np.concatenate([_block_edges(n, 900, 0, (0, 400), (0, 520), 1),
                        _block_edges(n, 900, 1, (384, 1024), (0, 300), 2)])
    graph = synth.Graph(n=n, edges=e, labels=["t0", "t1"], meta={"kind": "test"})
    g, q = tensor_parity(graph, "S A B\nA t0\nB t1\n", schedule=schedule, tensor_kind=kind)
    step = 128 if kind == eng.TENSOR_FP8 else 256
    occ_a = np.zeros((n // 128, n // step), dtype=bool)   # (m-tile, K step) of A
    occ_b = np.zeros((n // 256, n // step), dtype=bool)   # (n-tile, K step) of B^T
    a_e, b_e = e[e[:, 1] == 0], e[e[:, 1] == 1]
    occ_a[a_e[:, 0] // 128, a_e[:, 2] // step] = True
    occ_b[b_e[:, 2] // 256, b_e[:, 0] // step] = True
    live = int((occ_a.astype(np.int64) @ occ_b.T.astype(np.int64)).sum())
    s = q.stats()
    assert 0 < live < (n // 128) * (n // 256) * (n // step)
    assert s["tensor_live_ops"] == s["iterations"] * live * 2.0 * 128 * 256 * step


def _middle_restricted_graph(n, m, positions, seed):
    """S -> A B over A-edges i -> k and B-edges k -> j whose middle node k has k % 8 in
    `positions`: every K index of the product T_A x T_B that holds a one sits at one of those
    positions of its byte group."""
    ks = np.array([k for k in range(n) if k % 8 in positions], dtype=np.int64)
    kk = synth.key(seed, 9)
    i = np.arange(m, dtype=np.int64)
    a = np.stack([synth.uniform_int(kk, 4 * i, n), np.zeros(m, dtype=np.int64),
                  ks[synth.uniform_int(kk, 4 * i + 1, len(ks))]], axis=1)
    b = np.stack([ks[synth.uniform_int(kk, 4 * i + 2, len(ks))], np.ones(m, dtype=np.int64),
                  synth.uniform_int(kk, 4 * i + 3, n)], axis=1)
    return synth.Graph(n=n, edges=np.concatenate([a, b]), labels=["t0", "t1"], meta={"kind": "test"})


@KINDS
@pytest.mark.parametrize("positions", [(0,), (1,), (2,), (0, 1, 2), (3,), (6,), (7,), (3, 4, 5, 6, 7)],
                         ids=lambda p: "q" + "".join(map(str, p)))
@pytest.mark.parametrize("dense", [True, False])
def test_operand_encoding_positions(positions, dense, kind):
    """FP8: a one at K position q of a byte group (bit q + 8r of a 32-bit word) is the E4M3
    byte 1 << q (q = 0, 1, 2 are the subnormals 2^-9, 2^-8, 2^-7) and q = 7 is 0x40 = 2.0.
    FP4: a one at position s = q mod 4 of a nibble group (bit 4t + s) is the E2M1 nibble 1 << s
    (s = 0 is the subnormal 0.5) and s = 3 is 0b0100 = 2.0. A product is non-zero iff its
    accumulator is. If the MMA flushed subnormal inputs, or one position's encoding were wrong,
    the pairs whose only middle nodes sit at those positions would be lost. Each case puts
    every middle node at the given positions (530 nodes: several tiles and K stages plus a
    ragged tail) and compares with the oracle."""
    graph = _middle_restricted_graph(530, 1500, set(positions), seed=sum(positions) + 31 * len(positions))
    g, q = tensor_parity(graph, "S A B\nA t0\nB t1\n", schedule=eng.SCHED_JACOBI, dense_tensor=dense,
                         tensor_kind=kind)
    assert q.count("S") > 300
