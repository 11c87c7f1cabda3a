"""Sharded solve by row blocks (Section 7: the products of one loop execution on different
GPUs), checked on one device: every row block of one solve is a context of its own, all
driven from this process, exchanging their new pairs through the library's record export and
import (cfpq_block_*). Each block's context must end with the whole closure, equal to the
oracle's, after exactly Algorithm 1's Jacobi loop count."""
import ctypes

import numpy as np
import pytest
import torch

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng
from paper_1707_01007_b300 import shard

pytestmark = pytest.mark.gpu


def sharded(graph, text, parts, **kw):
    g = eng.Grammar(text, graph.labels)
    blocks = []
    for b0, b1 in shard.row_blocks(graph.n, parts):
        q = eng.Query(g, graph.n, graph.edges, schedule=eng.SCHED_JACOBI, row_begin=b0, row_end=b1,
                      timeout_s=120.0, **kw)
        blocks.append(shard.EngineBlock(q, b0, b1, len(g.names)))
    k = shard.solve_local(blocks)
    return g, [b.q for b in blocks], k


def check(graph, text, parts, **kw):
    g, qs, k = sharded(graph, text, parts, **kw)
    ref = oracle.hellings(graph, text)
    _, _, k_ref = oracle.matrix_closure_sparse(graph, text)
    assert k == k_ref
    for q in qs:
        assert q.stats()["iterations"] == k_ref
        for nm in g.names:
            assert np.array_equal(q.get(nm), ref.pairs(nm)), nm
    return g, qs


PATHS = [(eng.PATH_GATHER, {}), (eng.PATH_TENSOR, {}), (eng.PATH_TENSOR, {"dense_tensor": True}),
         (eng.PATH_TENSOR, {"tensor_kind": eng.TENSOR_FP8}), (eng.PATH_AUTO, {})]
PATH_IDS = ["gather", "tensor", "tensor-dense", "tensor-fp8", "auto"]


def test_row_blocks_split():
    assert shard.row_blocks(1000, 2) == [(0, 512), (512, 1000)]
    assert shard.row_blocks(3000, 3) == [(0, 1024), (1024, 2048), (2048, 3000)]
    assert shard.row_blocks(200, 4) == [(0, 200)]  # one 256-row unit: one block
    b = shard.row_blocks(16384, 8)
    assert b[0] == (0, 2048) and b[-1] == (14336, 16384) and all(x[1] == y[0] for x, y in zip(b, b[1:]))


@pytest.mark.parametrize("path,kw", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("parts", [2, 3])
def test_hierarchy_q1(path, kw, parts):
    check(synth.hierarchy(3000, 900, seed=4), synth.GRAMMAR_Q1, parts, path=path, **kw)


@pytest.mark.parametrize("path,kw", PATHS, ids=PATH_IDS)
def test_dense_closure(path, kw):
    # a dense transitive closure whose rows fill up: many rows of every block change in most
    # executions, and the right operand's rows come from every block
    check(synth.random_graph(1300, 2100, 1, seed=5), "S S S\nS t0\n", 3, path=path, **kw)


@pytest.mark.parametrize("path,kw", PATHS[:2], ids=PATH_IDS[:2])
def test_random_grammars(path, kw):
    for seed in range(3):
        graph = synth.random_graph(600 + 37 * seed, 1500, 3, seed=seed)
        text = synth.random_grammar_text(5, 3, 9, 6, seed % 3, seed=seed)
        check(graph, text, 2, path=path, **kw)


def test_two_cycles_across_blocks_jacobi_count():
    # two cycles of 9 and 8 nodes need 2pq + 1 = 145 executions; their nodes are spread over
    # 600 (v -> 37 v mod 600), so every step of a cycle may cross from one block to another
    base = synth.two_cycles(9, 8)
    e = np.asarray(base.edges, dtype=np.int64).copy()
    e[:, 0] = e[:, 0] * 37 % 600
    e[:, 2] = e[:, 2] * 37 % 600
    graph = synth.Graph(n=600, edges=e, labels=base.labels, meta={"kind": "test"})
    for path, kw in PATHS[:2]:
        g, qs = check(graph, synth.GRAMMAR_C3, 3, path=path, **kw)
        assert qs[0].stats()["iterations"] == 2 * 9 * 8 + 1


def test_hierarchy_full_size_tensor_two_blocks():
    # the benchmark's hierarchy at n = 16384, dense E2M1 tensor products, two row blocks
    check(synth.hierarchy(16384, 5000, seed=0), synth.GRAMMAR_QSC, 2, path=eng.PATH_TENSOR, dense_tensor=True)


def test_block_context_refuses_solve_and_batches():
    graph = synth.random_graph(600, 900, 2, seed=1)
    g = eng.Grammar("S A B\nA t0\nB t1\n", graph.labels)
    q = eng.Query(g, graph.n, graph.edges, schedule=eng.SCHED_JACOBI, row_begin=0, row_end=256)
    assert q.solve(check=False) == eng.ERR_INVALID
    with pytest.raises(eng.CfpqError) as ei:
        eng.solve_batch([q])
    assert ei.value.code == eng.ERR_INVALID
    with pytest.raises(eng.CfpqError) as ei:
        q.block_products()  # before cfpq_block_start
    assert ei.value.code == eng.ERR_NOT_SOLVED
    plain = eng.Query(g, graph.n, graph.edges)
    assert eng.library().cfpq_block_start(plain.handle, None) == eng.ERR_INVALID


def test_export_buffer_too_small_and_bad_records():
    graph = synth.random_graph(700, 3000, 2, seed=2)
    g = eng.Grammar("S A B\nA t0\nB t1\n", graph.labels)
    q = eng.Query(g, graph.n, graph.edges, schedule=eng.SCHED_JACOBI, row_begin=0, row_end=512)
    q.block_start()
    q.block_products()
    buf = torch.empty(q.record_words, dtype=torch.int32, device="cuda")
    with pytest.raises(eng.CfpqError) as ei:
        q.block_export(buf.data_ptr(), buf.numel())
    assert ei.value.code == eng.ERR_BUFFER and ei.value.words > q.record_words
    assert ei.value.words % q.record_words == 0
    # an imported record naming a non-terminal out of range is skipped and reported at the end
    bad = torch.zeros(q.record_words, dtype=torch.int32, device="cuda")
    bad[0] = 99
    with pytest.raises(eng.CfpqError) as ei:
        q.block_import(bad.data_ptr(), q.record_words - 1)  # not a whole number of records
    assert ei.value.code == eng.ERR_INVALID
    q.block_import(bad.data_ptr(), q.record_words)
    ch = ctypes.c_int32(7)
    assert eng.library().cfpq_block_finish(q.handle, None, ctypes.byref(ch)) == eng.ERR_INVALID
    assert ch.value == 0
