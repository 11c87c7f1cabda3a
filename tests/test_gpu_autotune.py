"""Batched-launch autotuner: every launch configuration (persistent grid size, gather tile
width per size class, schedule of CFPQ_SCHED_AUTO queries) gives the oracle's triples, and
the tuner installs the configuration it returns."""
import itertools

import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _restore_tuning():
    before = eng.batch_tuning()
    yield
    eng.set_batch_tuning(before)


def _batch(count, lo, hi, seed, schedules):
    work = synth.batch_queries(count, lo, hi, 0.3, seed=seed)
    out = []
    for j, (graph, text) in enumerate(work):
        g = eng.Grammar(text, graph.labels)
        out.append((graph, text, g, eng.Query(g, graph.n, graph.edges, path=eng.PATH_GATHER,
                                               schedule=schedules[j % len(schedules)])))
    return out


def _check_oracle(batch):
    for idx, (graph, text, g, q) in enumerate(batch):
        ref = oracle.hellings(graph, text)
        for nm in g.names:
            assert np.array_equal(q.get(nm), ref.pairs(nm)), (idx, nm)


def test_every_configuration_gives_the_oracle_result():
    # n from 64 to 3000: size classes 3 .. 7 (row lengths 8 .. 96 words)
    batch = _batch(20, 64, 3000, 11, [eng.SCHED_AUTO, eng.SCHED_INPLACE, eng.SCHED_JACOBI])
    qs = [q for *_, q in batch]
    expected = None
    for bps, cpl, sched in itertools.product([1, 2, 8], [1, 2, 4, 8], [eng.SCHED_INPLACE, eng.SCHED_JACOBI]):
        t = eng.batch_tuning_default()
        t.blocks_per_sm = bps
        for c in range(eng.TUNE_CLASSES):
            t.cpl[c] = cpl
            t.schedule[c] = sched
        eng.solve_batch(qs, tuning=t)
        got = [{nm: q.get(nm) for nm in g.names} for _, _, g, q in batch]
        if expected is None:
            _check_oracle(batch)
            expected = got
        else:
            for a, b in zip(expected, got):
                for nm in a:
                    assert np.array_equal(a[nm], b[nm]), (bps, cpl, sched, nm)


def test_auto_schedule_and_tile_follow_the_class_entry():
    # Jacobi runs exactly Algorithm 1's loop count (2pq + 1 on two cycles); an AUTO query
    # takes whichever schedule its size class holds, every query the class's tile width
    graph = synth.two_cycles(5, 4)
    g = eng.Grammar(synth.GRAMMAR_C3, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, path=eng.PATH_GATHER, schedule=eng.SCHED_AUTO)
    t = eng.batch_tuning_default()
    t.schedule[3] = eng.SCHED_JACOBI     # n_pad 256: W = 8, class 3
    t.cpl[3] = 4
    eng.solve_batch([q], tuning=t)
    st = q.stats()
    assert (st["schedule"], st["gather_cpl"], st["iterations"]) == (eng.SCHED_JACOBI, 4, 2 * 5 * 4 + 1)
    prof = eng.batch_last_profile()
    assert prof["rounds"] == 2 * 5 * 4 + 1      # one round per loop execution of the only query
    assert prof["products"] > 0 and prof["scan"] > 0 and prof["jacobi_merge"] > 0 and prof["start"] > 0
    assert sum(prof[k] for k in eng.BATCH_PHASES) <= st["solve_ms"] * 1.01
    assert len(prof["round_products"]) == 41 and abs(sum(prof["round_products"]) - prof["products"]) < 1e-3
    t.schedule[3] = eng.SCHED_INPLACE
    t.cpl[3] = 0                          # built-in: one word per lane for W <= 32
    eng.solve_batch([q], tuning=t)
    st = q.stats()
    assert (st["schedule"], st["gather_cpl"]) == (eng.SCHED_INPLACE, 1)
    assert q.count("S") == 5 * 4
    t.schedule[4] = eng.SCHED_JACOBI     # another class: no effect on this query
    eng.solve_batch([q], tuning=t)
    assert q.stats()["schedule"] == eng.SCHED_INPLACE
    # a single solve of an AUTO context is in place; explicit schedules are kept in batches
    q.solve()
    assert q.stats()["schedule"] == eng.SCHED_INPLACE
    qj = eng.Query(g, graph.n, graph.edges, path=eng.PATH_GATHER, schedule=eng.SCHED_JACOBI)
    eng.solve_batch([qj], tuning=t)
    assert (qj.stats()["schedule"], qj.stats()["iterations"]) == (eng.SCHED_JACOBI, 2 * 5 * 4 + 1)


def test_autotune_installs_its_choice_and_keeps_results():
    batch = _batch(40, 64, 4096, 2, [eng.SCHED_AUTO, eng.SCHED_INPLACE])
    qs = [q for *_, q in batch]
    best, rep = eng.autotune_batch(qs)
    assert rep["trials"] >= 2 and rep["default_ms"] > 0 and rep["best_ms"] > 0
    _check_oracle(batch)  # the contexts end with the chosen configuration's results
    installed = eng.batch_tuning()
    assert installed.blocks_per_sm == best.blocks_per_sm
    classes = {int(np.ceil(np.log2(((graph.n + 255) // 256 * 256) // 32))) for graph, *_ in batch}
    for c in classes:
        assert installed.cpl[c] == best.cpl[c]
    # the installed configuration is what cfpq_solve_batch now uses: same results again
    eng.solve_batch(qs)
    _check_oracle(batch)


def test_server_uses_installed_configuration():
    work = synth.batch_queries(16, 64, 2048, 0.3, seed=9)
    t = eng.batch_tuning_default()
    t.blocks_per_sm = 2
    for c in range(eng.TUNE_CLASSES):
        t.cpl[c] = 2
        t.schedule[c] = eng.SCHED_JACOBI
    eng.set_batch_tuning(t)
    srv = eng.Server(rounds_per_step=3)
    grammars = [eng.Grammar(text, graph.labels) for graph, text in work]
    tickets = [srv.submit(g, graph.n, graph.edges, schedule=eng.SCHED_AUTO) for g, (graph, _) in zip(grammars, work)]
    while srv.stats()["completed"] + srv.stats()["failed"] < len(work):
        srv.step()
    for tk, g, (graph, text) in zip(tickets, grammars, work):
        assert srv.info(tk)["status"] == eng.OK
        ref = oracle.hellings(graph, text)
        for nm in g.names:
            assert np.array_equal(srv.result(tk, g.id(nm)), ref.pairs(nm)), nm
    srv.close()


def test_tuned_solve_rejects_invalid_configuration():
    graph = synth.random_graph(40, 90, 2, seed=1)
    text = synth.random_grammar_text(4, 2, 7, 5, 0, seed=1)
    g = eng.Grammar(text, graph.labels)
    q = eng.Query(g, graph.n, graph.edges)
    t = eng.batch_tuning_default()
    t.cpl[3] = 3
    assert eng.solve_batch([q], tuning=t, check=False) == eng.ERR_INVALID


def _mixed_dense_batch():
    """Sparse hierarchy queries (n 64..1500) with block-diagonal closures of 2,048-8,192
    nodes (communities of 512, S -> S S | t0), all created on the automatic path."""
    out = []
    for graph, text in synth.batch_queries(24, 64, 1500, 0.3, seed=31):
        g = eng.Grammar(text, graph.labels)
        out.append((graph, text, g, eng.Query(g, graph.n, graph.edges)))
    for j, n in enumerate([2048, 3000, 4096, 6000, 8192]):
        graph = synth.communities(n, max(1, n // 512), 2, seed=40 + j)
        text = "S S S\nS t0\n"
        g = eng.Grammar(text, graph.labels)
        out.append((graph, text, g, eng.Query(g, graph.n, graph.edges)))
    return out


def test_classes_solved_alone_give_the_same_result():
    # the large classes leave the grouped launch (each query on its context's stream, with
    # the automatic product choice, tensor products included): same triples as grouped
    batch = _mixed_dense_batch()
    qs = [b[3] for b in batch]
    eng.solve_batch(qs, tuning=eng.batch_tuning_default())
    grouped = [{nm: q.get(nm) for nm in g.names} for _, _, g, q in batch]
    t = eng.batch_tuning_default()
    for c in range(6, eng.TUNE_CLASSES):
        t.product[c] = eng.BATCH_ALONE
    eng.solve_batch(qs, tuning=t)
    assert sum(q.stats()["tensor_products"] for q in qs) > 0  # the dense classes took the tensor cores
    for (graph, text, g, q), prev in zip(batch, grouped):
        for nm in g.names:
            assert np.array_equal(q.get(nm), prev[nm]), (graph.n, nm)
    _check_oracle(batch)


def test_autotune_solves_dense_large_classes_alone():
    batch = _mixed_dense_batch()
    qs = [b[3] for b in batch]
    best, report = eng.autotune_batch(qs)
    assert best.as_dict()["alone"], best.as_dict()
    assert report["best_ms"] < report["default_ms"]
    _check_oracle(batch)
