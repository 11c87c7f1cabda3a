"""Request loop for the continuous-batching server and its serial FIFO counterpart.

Both replay an arrival schedule (seconds from the start) in real time. The server loop
submits each query as soon as its arrival time has passed and calls ``Server.step()``
whenever work is queued or resident; the serial loop solves one query at a time in arrival
order with the single-query entry points. Latency = completion time - arrival time, where
completion means that every R_A of the query is in host memory.
"""
from __future__ import annotations

import time

import numpy as np

from . import PATH_GATHER, Query, Server


def _summary(arrivals, done_at, t_end):
    lat = np.asarray(done_at) - np.asarray(arrivals)
    span = max(t_end - float(arrivals[0]), 1e-9)
    return {"queries": len(arrivals), "queries_per_s": len(arrivals) / span,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "makespan_s": span}


def run_server(server: Server, queries, arrivals, keep_results: bool = False):
    """queries: list of (Grammar, n, edges). Returns (summary, results) where results[i] is
    {name: (k, 2) array} when keep_results, else None."""
    n_q = len(queries)
    order = np.argsort(arrivals, kind="stable")
    arrivals = np.asarray(arrivals, dtype=np.float64)
    done_at = np.zeros(n_q)
    results = [None] * n_q
    tickets = {}
    i = done = 0
    t0 = time.perf_counter()
    while done < n_q:
        now = time.perf_counter() - t0
        while i < n_q and arrivals[order[i]] <= now:
            j = int(order[i])
            g, n, e = queries[j]
            tickets[server.submit(g, n, e)] = j
            i += 1
        st = server.stats()
        if st["queued"] + st["resident"] > 0:
            server.step()
            t = time.perf_counter() - t0
            for tk in server.completed():
                j = tickets[tk]
                done_at[j] = t
                if keep_results:
                    info = server.info(tk)
                    g = queries[j][0]
                    results[j] = {nm: server.result(tk, a) for a, nm in enumerate(g.names)} \
                        if info["state"] == 2 else info
                server.release(tk)
                done += 1
        elif i < n_q:
            time.sleep(max(0.0, arrivals[order[i]] - now))
    t_end = time.perf_counter() - t0
    return _summary(arrivals, done_at, t_end), results


def run_serial(queries, arrivals):
    """One query at a time in arrival order (create, solve, copy every R_A back with one
    call, destroy)."""
    n_q = len(queries)
    order = np.argsort(arrivals, kind="stable")
    arrivals = np.asarray(arrivals, dtype=np.float64)
    done_at = np.zeros(n_q)
    t0 = time.perf_counter()
    for j in order:
        now = time.perf_counter() - t0
        if arrivals[j] > now:
            time.sleep(arrivals[j] - now)
        g, n, e = queries[j]
        q = Query(g, n, e, path=PATH_GATHER)
        q.solve()
        q.triples_all()
        q.close()
        done_at[j] = time.perf_counter() - t0
    return _summary(arrivals, done_at, time.perf_counter() - t0)
