"""Serving (continuous batching): every query's result equals its oracle result and its
result when solved alone; admission never exceeds the HBM budget."""
import numpy as np
import pytest

import cfpq_synth as synth
import oracle
import paper_1707_01007_b300 as eng
from paper_1707_01007_b300 import serve

pytestmark = pytest.mark.gpu


def _work(count, n_lo, n_hi, seed):
    out = []
    for graph, text in synth.batch_queries(count, n_lo, n_hi, 0.3, seed=seed):
        out.append((graph, text, eng.Grammar(text, graph.labels)))
    return out


def test_server_results_equal_oracle_and_alone():
    work = _work(40, 64, 1500, seed=11)
    srv = eng.Server(rounds_per_step=2)
    tickets = [srv.submit(g, graph.n, graph.edges) for graph, text, g in work]
    while srv.stats()["completed"] + srv.stats()["failed"] < len(work):
        srv.step()
    for tk, (graph, text, g) in zip(tickets, work):
        info = srv.info(tk)
        assert info["state"] == eng.QUERY_DONE and info["status"] == eng.OK
        ref = oracle.hellings(graph, text)
        alone = eng.Query(g, graph.n, graph.edges, path=eng.PATH_GATHER)
        alone.solve()
        for a, nm in enumerate(g.names):
            got = srv.result(tk, a)
            assert np.array_equal(got, ref.pairs(nm)), nm
            assert np.array_equal(got, alone.get(nm))
    srv.close()


def test_admission_respects_budget_and_rejects_too_large():
    work = _work(24, 256, 2048, seed=12)
    biggest = max(graph.n for graph, _, _ in work)
    plane = (biggest + 255) // 256 * 256
    budget = int(3 * 7 * plane * plane / 8 * 1.6) + (1 << 20)
    srv = eng.Server(hbm_budget_bytes=budget, rounds_per_step=3)
    tickets = [srv.submit(g, graph.n, graph.edges) for graph, text, g in work]
    huge = synth.hierarchy(16384, 5000, seed=1)
    g_huge = eng.Grammar(synth.GRAMMAR_Q1, huge.labels)
    t_huge = srv.submit(g_huge, huge.n, huge.edges)
    while srv.stats()["completed"] + srv.stats()["failed"] < len(work) + 1:
        srv.step()
        st = srv.stats()
        assert st["used_bytes"] <= st["budget_bytes"]
    st = srv.stats()
    assert st["peak_used_bytes"] <= budget and st["failed"] == 1
    info = srv.info(t_huge)
    assert info["state"] == eng.QUERY_FAILED and info["status"] == eng.ERR_NOMEM
    for tk, (graph, text, g) in zip(tickets, work):
        ref = oracle.hellings(graph, text)
        for a, nm in enumerate(g.names):
            assert np.array_equal(srv.result(tk, a), ref.pairs(nm))
    srv.close()


def test_stream_with_arrivals_and_mixed_schedules():
    work = _work(30, 64, 1024, seed=13)
    queries = [(g, graph.n, graph.edges) for graph, text, g in work]
    arrivals = synth.poisson_arrivals(len(queries), rate_per_s=2000.0, seed=13)
    srv = eng.Server(rounds_per_step=4)
    summary, results = serve.run_server(srv, queries, arrivals, keep_results=True)
    assert summary["queries"] == 30 and summary["p99_ms"] >= summary["p50_ms"] > 0
    for (graph, text, g), res in zip(work, results):
        ref = oracle.hellings(graph, text)
        for nm in g.names:
            assert np.array_equal(res[nm], ref.pairs(nm))
    srv.close()


def test_ticket_errors():
    srv = eng.Server()
    with pytest.raises(eng.CfpqError):
        srv.info(12345)
    graph = synth.hierarchy(300, 90, seed=2)
    g = eng.Grammar(synth.GRAMMAR_QSC, graph.labels)
    tk = srv.submit(g, graph.n, graph.edges)
    with pytest.raises(eng.CfpqError):
        srv.result(tk, 0)          # not solved yet
    while srv.info(tk)["state"] != eng.QUERY_DONE:
        srv.step()
    srv.result(tk, 0)
    srv.release(tk)
    with pytest.raises(eng.CfpqError):
        srv.info(tk)
    srv.close()


def test_large_queries_run_alone_beside_the_grouped_launches():
    """Queries with at least 16,384 (padded) rows are solved by the single-query loop on the
    server's second stream while the small ones go through the grouped launches: every
    result still equals the oracle's and the query's result when solved alone."""
    small = _work(30, 64, 2000, seed=21)
    big = [(synth.hierarchy(n, round(0.3 * n), seed=n), text) for n, text in
           [(16384, synth.GRAMMAR_Q1), (20000, synth.GRAMMAR_QSC), (16000, synth.GRAMMAR_Q1)]]
    work = small[:10] + [(gr, t, eng.Grammar(t, gr.labels)) for gr, t in big[:2]] + small[10:20] + \
        [(big[2][0], big[2][1], eng.Grammar(big[2][1], big[2][0].labels))] + small[20:]
    srv = eng.Server(rounds_per_step=4)
    tickets = []
    for j, (graph, text, g) in enumerate(work):
        tickets.append(srv.submit(g, graph.n, graph.edges))
        if j % 5 == 4:
            srv.step()  # arrivals while others are resident
    while srv.stats()["completed"] + srv.stats()["failed"] < len(work):
        srv.step()
    for tk, (graph, text, g) in zip(tickets, work):
        info = srv.info(tk)
        assert info["state"] == eng.QUERY_DONE and info["status"] == eng.OK, graph.n
        ref = oracle.hellings(graph, text)
        alone = eng.Query(g, graph.n, graph.edges, path=eng.PATH_GATHER)
        alone.solve()
        for a, nm in enumerate(g.names):
            got = srv.result(tk, a)
            assert np.array_equal(got, ref.pairs(nm)), (graph.n, nm)
            assert np.array_equal(got, alone.get(nm))
        srv.release(tk)
    srv.close()
