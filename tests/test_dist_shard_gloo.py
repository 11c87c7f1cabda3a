"""The sharded loop's exchange on CPU: two or three gloo ranks (127.0.0.1) run
shard.solve_sharded, each with its own row block, and all-gather their records with
shard.TorchExchange. The per-block product is a test stand-in (dense NumPy Boolean matrices
over the oracle's grammar reader, restricted to the block's rows) that speaks the engine's
record format: [A, i, the W = n_pad / 32 words of row i's new pairs]. Every rank must end
with the oracle's closure after Algorithm 1's Jacobi loop count (Section 4.2)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class NumpyBlock:
    """Test stand-in for one rank's row block: one Jacobi step of Algorithm 1 on dense
    Boolean matrices, the products computing rows [r0, r1) only."""

    def __init__(self, graph, text, r0, r1):
        import oracle
        import torch

        self.torch = torch
        self.cnf = oracle.parse_grammar(text, graph.labels)
        self.graph, self.r0, self.r1 = graph, r0, r1
        self.n = graph.n
        self.n_pad = (self.n + 255) // 256 * 256
        self.W = self.n_pad // 32
        self.nt = len(self.cnf.names)

    def start(self):
        n = self.n
        self.T = np.zeros((self.nt, n, n), dtype=bool)
        for s, lab, d in np.asarray(self.graph.edges, dtype=np.int64):
            for a, x in self.cnf.unary:
                if x == lab:
                    self.T[a, s, d] = True
        for a in self.cnf.eps:
            self.T[a][np.arange(n), np.arange(n)] = True
        self.inbox = np.zeros_like(self.T)

    def products(self):
        r0, r1 = self.r0, self.r1
        self.N = np.zeros((self.nt, r1 - r0, self.n), dtype=bool)
        for a, b, c in self.cnf.binary:
            p = (self.T[b, r0:r1].astype(np.int64) @ self.T[c].astype(np.int64)) > 0
            self.N[a] |= p & ~self.T[a, r0:r1]

    def _pack(self, row):
        bits = np.zeros(self.n_pad, dtype=bool)
        bits[: self.n] = row
        return np.packbits(bits, bitorder="little").view("<u4")

    def export(self):
        recs = []
        for a in range(self.nt):
            for k in np.flatnonzero(self.N[a].any(axis=1)):
                recs.append(np.concatenate([np.array([a, self.r0 + k], dtype="<u4"), self._pack(self.N[a, k])]))
        flat = np.concatenate(recs).view(np.int32) if recs else np.zeros(1, dtype=np.int32)
        return self.torch.from_numpy(flat.copy()), sum(len(r) for r in recs)

    def import_(self, records, words):
        rec_words = 2 + self.W
        arr = records[:words].numpy().view("<u4").reshape(-1, rec_words)
        for r in arr:
            a, i = int(r[0]), int(r[1])
            bits = np.unpackbits(r[2:].view(np.uint8), bitorder="little")[: self.n].astype(bool)
            self.inbox[a, i] |= bits

    def finish(self):
        changed = bool(self.N.any() or self.inbox.any())
        self.T[:, self.r0:self.r1] |= self.N
        self.T |= self.inbox
        self.inbox[:] = False
        return changed


def _rank_main(rank, world, port, case, out):
    sys.path.insert(0, ROOT)
    import cfpq_synth as synth
    from paper_1707_01007_b300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        graph, text = case(synth)
        blocks = shard.row_blocks(graph.n, world)
        r0, r1 = blocks[rank]
        block = NumpyBlock(graph, text, r0, r1)
        k = shard.solve_sharded(block, shard.TorchExchange("cpu"), max_executions=10000)
        out.put((rank, k, {nm: np.argwhere(block.T[a]).astype(np.uint32) for a, nm in enumerate(block.cnf.names)}))
    finally:
        dist.destroy_process_group()


def _hierarchy(synth):
    return synth.hierarchy(700, 200, seed=3), synth.GRAMMAR_Q1


def _dense(synth):
    return synth.random_graph(600, 900, 1, seed=2), "S S S\nS t0\n"


def _cycles(synth):
    base = synth.two_cycles(6, 5)
    e = np.asarray(base.edges, dtype=np.int64).copy()
    e[:, 0] = e[:, 0] * 101 % 530
    e[:, 2] = e[:, 2] * 101 % 530
    return synth.Graph(n=530, edges=e, labels=base.labels, meta={"kind": "test"}), synth.GRAMMAR_C3


@pytest.mark.parametrize("case,world", [(_hierarchy, 2), (_dense, 2), (_cycles, 3)],
                         ids=["hierarchy-2", "dense-2", "cycles-3"])
def test_gloo_ranks_reach_the_oracle_closure(case, world):
    sys.path.insert(0, ROOT)
    import cfpq_synth as synth
    import oracle

    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = [out.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    graph, text = case(synth)
    ref = oracle.hellings(graph, text)
    _, _, k_ref = oracle.matrix_closure_sparse(graph, text)
    for rank, k, rel in got:
        assert k == k_ref, rank
        for nm, pairs in rel.items():
            assert np.array_equal(pairs, ref.pairs(nm)), (rank, nm)


def test_row_blocks_cover_the_rows_once():
    sys.path.insert(0, ROOT)
    from paper_1707_01007_b300 import shard

    for n in (1, 255, 256, 257, 1000, 16384, 65535, 131072):
        for parts in (1, 2, 3, 8):
            b = shard.row_blocks(n, parts)
            assert b[0][0] == 0 and b[-1][1] == n and len(b) <= parts
            assert all(x[1] == y[0] and x[1] % 256 == 0 for x, y in zip(b, b[1:]))
            assert all(x[0] < x[1] for x in b)
