"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every entry
point ``include/cfpq.h`` declares, rejects invalid input before touching the device, and
its grammar reader produces the same normal form as the oracle's independent reader."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names |= set(re.findall(r"\b(cfpq_[a-z_]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = eng.library()
    decl = declared_functions()
    assert len(decl) >= 14
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(eng.EXPORTS) == decl


def test_strerror_names_every_status():
    lib = eng.library()
    names = {lib.cfpq_strerror(c).decode() for c in range(10)}
    assert len(names) == 10
    assert lib.cfpq_strerror(99).decode() == "unknown status"


@pytest.mark.parametrize("text,labels", [
    (synth.GRAMMAR_Q1, synth.HIERARCHY_LABELS),
    (synth.GRAMMAR_QSC, synth.HIERARCHY_LABELS),
    (synth.GRAMMAR_C3, ["a", "b"]),
    (synth.GRAMMAR_WORKED, synth.HIERARCHY_LABELS),
    (synth.GRAMMAR_Q2, synth.HIERARCHY_LABELS),
    (synth.random_grammar_text(6, 3, 12, 8, 2, seed=5), ["t0", "t1", "t2"]),
    ("S a S1\nS1 S b\nS a b\n", ["a", "b"]),
])
def test_grammar_reader_matches_oracle_reader(text, labels):
    g = eng.Grammar(text, labels)
    c = oracle.parse_grammar(text, labels)
    assert g.names == c.names
    cn = g.cnf.contents
    assert [(cn.unary[i].lhs, cn.unary[i].term) for i in range(cn.n_unary)] == list(map(tuple, c.unary))
    assert [(cn.binary[i].lhs, cn.binary[i].b, cn.binary[i].c) for i in range(cn.n_binary)] == \
        list(map(tuple, c.binary))
    assert [cn.eps_lhs[i] for i in range(cn.n_eps)] == list(c.eps)


@pytest.mark.parametrize("text", ["S A\nA a\n", "S zz\n", "S a b c\n", "eps a\n", "S <a>\n"])
def test_grammar_reader_rejects(text):
    with pytest.raises(ValueError):
        eng.Grammar(text, ["a", "b", "c"])


def _create(cnf, n, edges, opt=None):
    rec = np.zeros(len(edges), dtype=[("src", "<u4"), ("label", "<i4"), ("dst", "<u4")])
    for i, (s, l, d) in enumerate(edges):
        rec[i] = (s, l, d)
    h = ctypes.c_void_p()
    ptr = rec.ctypes.data_as(ctypes.POINTER(eng.Edge)) if len(edges) else None
    return eng.library().cfpq_create(cnf, n, ptr, len(edges), opt, ctypes.byref(h)), h


def test_create_rejects_invalid_input_before_device_use():
    g = eng.Grammar("S S S\nS a\n", ["a"])
    assert _create(g.cnf, 0, [])[0] == eng.ERR_INVALID                  # n = 0
    assert _create(g.cnf, 4, [(0, 0, 9)])[0] == eng.ERR_INVALID         # dst >= n
    assert _create(g.cnf, 4, [(0, 3, 1)])[0] == eng.ERR_INVALID         # label out of range
    assert _create(g.cnf, 200000, [])[0] == eng.ERR_INVALID             # n > CFPQ_MAX_NODES
    bad = eng.GrammarCNF()
    bad.n_nonterm, bad.n_term = 1, 1
    r1 = (eng.Rule1 * 1)(eng.Rule1(3, 0))                               # lhs out of range
    bad.unary, bad.n_unary = r1, 1
    assert _create(ctypes.pointer(bad), 4, [])[0] == eng.ERR_INVALID
    opt = eng.Options()
    eng.library().cfpq_options_default(ctypes.byref(opt))
    opt.schedule = 7
    assert _create(g.cnf, 4, [], ctypes.byref(opt))[0] == eng.ERR_INVALID


def test_lengths_options_checked_before_device_use():
    # single-path lengths (Section 5) come from the matrices before each loop execution, so
    # they need the Jacobi schedule and a matrix path; bad flag values are rejected
    g = eng.Grammar("S S S\nS a\n", ["a"])
    lib = eng.library()
    for field, value, code in [("lengths", 2, eng.ERR_INVALID), ("dense_tensor", 2, eng.ERR_INVALID),
                               ("tensor_kind", 3, eng.ERR_INVALID), ("tensor_kind", -1, eng.ERR_INVALID)]:
        opt = eng.Options()
        lib.cfpq_options_default(ctypes.byref(opt))
        opt.schedule = eng.SCHED_JACOBI
        setattr(opt, field, value)
        assert _create(g.cnf, 4, [(0, 0, 1)], ctypes.byref(opt))[0] == code, field
    for schedule, path in [(eng.SCHED_INPLACE, eng.PATH_GATHER), (eng.SCHED_JACOBI, eng.PATH_WORKLIST)]:
        opt = eng.Options()
        lib.cfpq_options_default(ctypes.byref(opt))
        opt.schedule, opt.path, opt.lengths = schedule, path, 1
        assert _create(g.cnf, 4, [(0, 0, 1)], ctypes.byref(opt))[0] == eng.ERR_UNSUPPORTED
    assert lib.cfpq_get_lengths(None, 0, None, None, 0, None) == eng.ERR_INVALID
    # row blocks of a sharded solve: 256-aligned ends inside [0, n], Jacobi on a matrix path
    for b0, b1, code in [(100, 600, eng.ERR_INVALID), (0, 700, eng.ERR_INVALID), (512, 256, eng.ERR_INVALID),
                         (256, 256, eng.ERR_INVALID), (0, 300, eng.ERR_INVALID)]:
        opt = eng.Options()
        lib.cfpq_options_default(ctypes.byref(opt))
        opt.schedule, opt.row_begin, opt.row_end = eng.SCHED_JACOBI, b0, b1
        assert _create(g.cnf, 600, [(0, 0, 1)], ctypes.byref(opt))[0] == code, (b0, b1)
    for schedule, path in [(eng.SCHED_INPLACE, eng.PATH_GATHER), (eng.SCHED_JACOBI, eng.PATH_WORKLIST)]:
        opt = eng.Options()
        lib.cfpq_options_default(ctypes.byref(opt))
        opt.schedule, opt.path, opt.row_begin, opt.row_end = schedule, path, 256, 600
        assert _create(g.cnf, 600, [(0, 0, 1)], ctypes.byref(opt))[0] == eng.ERR_UNSUPPORTED
    for name in ("cfpq_block_start", "cfpq_block_products"):
        assert getattr(lib, name)(None, None) == eng.ERR_INVALID
    assert lib.cfpq_block_export(None, None, 0, None, None) == eng.ERR_INVALID
    assert lib.cfpq_block_import(None, None, 0, None) == eng.ERR_INVALID
    assert lib.cfpq_block_finish(None, None, None) == eng.ERR_INVALID
    assert lib.cfpq_state_size(None, None) == eng.ERR_INVALID
    assert lib.cfpq_export_state(None, None, 0) == eng.ERR_INVALID
    assert lib.cfpq_import_state(None, None, 0) == eng.ERR_INVALID
    assert lib.cfpq_resume(None, None, 0) == eng.ERR_INVALID
    assert lib.cfpq_get_path(None, 0, 0, 0, None, None, 0, None) == eng.ERR_INVALID


def test_null_arguments():
    lib = eng.library()
    assert lib.cfpq_solve(None, None) == eng.ERR_INVALID
    assert lib.cfpq_get(None, 0, None, 0, None) == eng.ERR_INVALID
    assert lib.cfpq_get_device(None, 0, None, 0, None) == eng.ERR_INVALID
    assert lib.cfpq_get_all_device(None, None, 0, None) == eng.ERR_INVALID
    assert lib.cfpq_count(None, 0, None) == eng.ERR_INVALID
    assert lib.cfpq_stats_get(None, None) == eng.ERR_INVALID
    assert lib.cfpq_options_default(None) == eng.ERR_INVALID
    assert lib.cfpq_solve_batch(None, 0, None) == eng.ERR_INVALID
    assert lib.cfpq_measure_mma_sync_peaks(None, None) == eng.ERR_INVALID
    assert lib.cfpq_measure_tensor_peaks(None) == eng.ERR_INVALID
    lib.cfpq_destroy(None)


def test_options_defaults():
    opt = eng.Options()
    assert eng.library().cfpq_options_default(ctypes.byref(opt)) == eng.OK
    assert (opt.schedule, opt.path, opt.use_graph, opt.profile, opt.max_iter, opt.lengths, opt.dense_tensor,
            opt.tensor_kind) == (eng.SCHED_INPLACE, eng.PATH_AUTO, 1, 0, 0, 0, 0, eng.TENSOR_AUTO)
    assert ctypes.sizeof(eng.Options) == 56


def test_batch_tuning_host_calls():
    lib = eng.library()
    d = eng.batch_tuning_default()
    assert d.blocks_per_sm == 0 and all(v == 0 for v in d.cpl) and all(v == eng.SCHED_INPLACE for v in d.schedule)
    before = eng.batch_tuning()
    try:
        t = eng.batch_tuning_default()
        t.blocks_per_sm = 4
        t.cpl[5], t.cpl[9] = 2, 8
        t.schedule[7] = eng.SCHED_JACOBI
        eng.set_batch_tuning(t)
        got = eng.batch_tuning()
        assert got.as_dict() == {"blocks_per_sm": 4, "cpl": {5: 2, 9: 8}, "schedule": {7: eng.SCHED_JACOBI},
                                 "alone": []}
        t.product[11] = eng.BATCH_ALONE
        eng.set_batch_tuning(t)
        got = eng.batch_tuning()
        assert got.as_dict()["alone"] == [11]
        # every invalid field is rejected and leaves the installed configuration unchanged
        for field, idx, value in [("blocks_per_sm", None, 9), ("blocks_per_sm", None, -1), ("cpl", 3, 3),
                                  ("cpl", 4, 16), ("schedule", 6, eng.SCHED_AUTO), ("schedule", 2, -1),
                                  ("product", 8, 2), ("product", 3, -1)]:
            bad = eng.batch_tuning_default()
            if idx is None:
                setattr(bad, field, value)
            else:
                getattr(bad, field)[idx] = value
            assert lib.cfpq_batch_tuning_set(ctypes.byref(bad)) == eng.ERR_INVALID, (field, idx, value)
            assert eng.batch_tuning().as_dict() == got.as_dict()
        assert lib.cfpq_batch_tuning_set(None) == eng.ERR_INVALID
        assert lib.cfpq_batch_tuning_get(None) == eng.ERR_INVALID
        assert lib.cfpq_autotune_batch(None, 0, None, None, None) == eng.ERR_INVALID
        assert lib.cfpq_solve_batch_tuned(None, 0, ctypes.byref(t), None) == eng.ERR_INVALID
    finally:
        eng.set_batch_tuning(before)



def test_batch_profile_host_call():
    lib = eng.library()
    assert lib.cfpq_batch_last_profile(None, 3, None, None, 0) == eng.ERR_INVALID
    assert lib.cfpq_batch_last_profile(None, 0, None, None, 2) == eng.ERR_INVALID
    assert lib.cfpq_batch_last_profile(None, 0, None, None, 0) == eng.OK
    p = eng.batch_last_profile()
    assert list(p)[:len(eng.BATCH_PHASES)] == list(eng.BATCH_PHASES) and p["rounds"] >= 0
