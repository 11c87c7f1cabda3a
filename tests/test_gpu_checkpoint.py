"""Checkpoint and resume of the fixpoint loop: a solve stopped after k executions of
Algorithm 1's loop (Section 4.2), its state exported, imported into a fresh context and
resumed, ends with the same relations as an uninterrupted solve (the oracle's: the closure
is monotone with a unique least fixpoint, Theorem 2), and under the Jacobi schedule after
the same total number of executions."""
import ctypes

import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu

PATHS = [(eng.PATH_GATHER, eng.SCHED_JACOBI, {}), (eng.PATH_GATHER, eng.SCHED_INPLACE, {}),
         (eng.PATH_TENSOR, eng.SCHED_JACOBI, {"dense_tensor": True}), (eng.PATH_TENSOR, eng.SCHED_INPLACE, {}),
         (eng.PATH_AUTO, eng.SCHED_JACOBI, {}), (eng.PATH_AUTO, eng.SCHED_INPLACE, {})]
IDS = ["gather-jacobi", "gather-inplace", "tensor-dense-jacobi", "tensor-inplace", "auto-jacobi", "auto-inplace"]


def _query(graph, text, path, schedule, **kw):
    g = eng.Grammar(text, graph.labels)
    return g, eng.Query(g, graph.n, graph.edges, path=path, schedule=schedule, timeout_s=120.0, **kw)


def _same_as_oracle(g, q, graph, text):
    ref = oracle.hellings(graph, text)
    for nm in g.names:
        assert np.array_equal(q.get(nm), ref.pairs(nm)), nm


@pytest.mark.parametrize("path,schedule,kw", PATHS, ids=IDS)
@pytest.mark.parametrize("case", ["hierarchy", "cycles"])
def test_stop_export_import_resume(path, schedule, kw, case):
    if case == "hierarchy":
        graph, text, stop = synth.hierarchy(3000, 900, seed=6), synth.GRAMMAR_Q1, 4
    else:
        graph, text, stop = synth.two_cycles(9, 8), synth.GRAMMAR_C3, 50
    g, q1 = _query(graph, text, path, schedule, max_iter=stop, **kw)
    assert q1.solve(check=False) == eng.ERR_ITER_LIMIT
    assert q1.stats()["iterations"] == stop
    image = q1.export_state()
    _, q2 = _query(graph, text, path, schedule, **kw)
    q2.import_state(image)
    q2.resume()
    _same_as_oracle(g, q2, graph, text)
    if schedule == eng.SCHED_JACOBI:
        _, _, k = oracle.matrix_closure_sparse(graph, text)
        assert q2.stats()["iterations"] == k


@pytest.mark.parametrize("path,schedule,kw", PATHS[:2] + PATHS[4:5], ids=IDS[:2] + IDS[4:5])
def test_resume_in_place_and_in_stages(path, schedule, kw):
    graph, text = synth.two_cycles(9, 8), synth.GRAMMAR_C3
    g, q = _query(graph, text, path, schedule, max_iter=20, **kw)
    assert q.solve(check=False) == eng.ERR_ITER_LIMIT
    assert q.resume(more_executions=30, check=False) == eng.ERR_ITER_LIMIT  # 50 executions so far
    image = q.export_state()
    _, q2 = _query(graph, text, path, schedule, **kw)
    q2.import_state(image)
    assert q2.resume(more_executions=40, check=False) == eng.ERR_ITER_LIMIT  # 90
    q2.resume()  # the rest, on the resumed context
    _same_as_oracle(g, q2, graph, text)
    if schedule == eng.SCHED_JACOBI:
        assert q2.stats()["iterations"] == 2 * 9 * 8 + 1
    q.resume()  # the first context goes on from 50 by itself
    _same_as_oracle(g, q, graph, text)


def test_full_size_hierarchy_checkpoint():
    graph = synth.hierarchy(16384, 5000, seed=0)
    g, q = _query(graph, synth.GRAMMAR_Q1, eng.PATH_TENSOR, eng.SCHED_JACOBI, max_iter=7)
    assert q.solve(check=False) == eng.ERR_ITER_LIMIT
    image = q.export_state()
    _, q2 = _query(graph, synth.GRAMMAR_Q1, eng.PATH_AUTO, eng.SCHED_JACOBI)  # another product path
    q2.import_state(image)
    q2.resume()
    _same_as_oracle(g, q2, graph, synth.GRAMMAR_Q1)


def test_statuses():
    graph = synth.hierarchy(700, 200, seed=1)
    g, q = _query(graph, synth.GRAMMAR_Q1, eng.PATH_GATHER, eng.SCHED_JACOBI, max_iter=3)
    lib = eng.library()
    buf = np.zeros(64, dtype=np.uint8)
    assert lib.cfpq_export_state(q.handle, buf.ctypes.data_as(ctypes.c_void_p), buf.size) == eng.ERR_NOT_SOLVED
    assert lib.cfpq_resume(q.handle, None, 0) == eng.ERR_NOT_SOLVED
    assert q.solve(check=False) == eng.ERR_ITER_LIMIT
    assert lib.cfpq_export_state(q.handle, buf.ctypes.data_as(ctypes.c_void_p), buf.size) == eng.ERR_BUFFER
    image = q.export_state()
    # an image fits only a context of the same shape and grammar
    other_n = synth.hierarchy(800, 200, seed=1)
    _, q_n = _query(other_n, synth.GRAMMAR_Q1, eng.PATH_GATHER, eng.SCHED_JACOBI)
    _, q_g = _query(graph, synth.GRAMMAR_QSC, eng.PATH_GATHER, eng.SCHED_JACOBI)
    for qq in (q_n, q_g):
        with pytest.raises(eng.CfpqError) as ei:
            qq.import_state(image)
        assert ei.value.code == eng.ERR_INVALID
    broken = image.copy()
    broken[0] ^= 0xFF
    _, q3 = _query(graph, synth.GRAMMAR_Q1, eng.PATH_GATHER, eng.SCHED_JACOBI)
    with pytest.raises(eng.CfpqError) as ei:
        q3.import_state(broken)
    assert ei.value.code == eng.ERR_INVALID
    with pytest.raises(eng.CfpqError) as ei:
        q3.import_state(image[:-1])
    assert ei.value.code == eng.ERR_INVALID
    # worklist and lengths contexts have no such state
    cyc = synth.two_cycles(5, 4)
    _, qw = _query(cyc, synth.GRAMMAR_C3, eng.PATH_WORKLIST, eng.SCHED_INPLACE)
    n = ctypes.c_size_t()
    assert lib.cfpq_state_size(qw.handle, ctypes.byref(n)) == eng.ERR_UNSUPPORTED
    gl = eng.Grammar(synth.GRAMMAR_Q1, graph.labels)
    ql = eng.Query(gl, graph.n, graph.edges, schedule=eng.SCHED_JACOBI, lengths=True)
    assert lib.cfpq_state_size(ql.handle, ctypes.byref(n)) == eng.ERR_UNSUPPORTED
    # a finished solve has nothing to resume
    q.resume()
    assert lib.cfpq_resume(q.handle, None, 0) == eng.ERR_NOT_SOLVED
