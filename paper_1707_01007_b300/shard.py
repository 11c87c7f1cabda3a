"""Sharded solve by row blocks: the loop of Algorithm 1 (Section 4.2) spread over ranks.

The paper's remark on parallelism (Section 7) is that the matrix products of one loop
execution may run on different GPUs independently. Here rank r owns a block of rows
[b_r, b_{r+1}) of every T_A. Its context computes those rows of every product T_B x T_C,
which needs those rows of T_B and all of T_C, so every rank keeps all of T. One loop
execution is:

    products over the rank's rows  ->  exchange of the new pairs  ->  merge on every rank

The exchange is an all-gather of variable-size records (cfpq_block_export): each rank sends
the rows to which its products added pairs, and imports everyone else's (cfpq_block_import).
Every rank then merges the same union, so all ranks hold the same T_k after k executions
and stop at the same execution (Jacobi schedule). The records travel by torch.distributed:
device tensors under NCCL, host tensors under gloo. No kernel reads another rank's memory
or waits for another rank.

    blocks = row_blocks(n, world)
    q = Query(g, n, edges, schedule=SCHED_JACOBI, row_begin=blocks[rank][0], row_end=blocks[rank][1])
    solve_sharded(EngineBlock(q, device), TorchExchange(device))
    q.get("S")          # every rank holds the whole closure
"""
from __future__ import annotations

from . import Query


def row_blocks(n: int, parts: int):
    """[begin, end) row blocks of an n-node query for `parts` ranks: 256-aligned boundaries
    (the row tiling of the product kernels), as even as that allows, the last ending at n.
    Fewer blocks than parts when n is small (a rank with no block has nothing to compute)."""
    if n <= 0 or parts <= 0:
        raise ValueError("n and parts must be positive")
    units = (n + 255) // 256
    parts = min(parts, units)
    out, u0 = [], 0
    for p in range(parts):
        u1 = u0 + units // parts + (1 if p < units % parts else 0)
        out.append((u0 * 256, min(u1 * 256, n)))
        u0 = u1
    return out


class EngineBlock:
    """One rank's row block on the engine: a Query created with row_begin / row_end and a
    device buffer for its outgoing records (sized for every row of the block flagged)."""

    def __init__(self, query: Query, row_begin: int, row_end: int, n_nonterm: int, device="cuda"):
        import torch

        self.q = query
        self.torch = torch
        self.device = torch.device(device)
        self.rec_words = query.record_words
        cap = max(1, (row_end - row_begin) * n_nonterm * self.rec_words)
        self.buf = torch.empty(cap, dtype=torch.int32, device=self.device)

    def start(self):
        self.q.block_start()

    def products(self):
        self.q.block_products()

    def export(self):
        """(tensor, words): this execution's records of the block's rows."""
        words = self.q.block_export(self.buf.data_ptr(), self.buf.numel())
        return self.buf, words

    def import_(self, records, words: int):
        if words == 0:
            return
        if records.device != self.device:
            records = records[:words].to(self.device)
        self.q.block_import(records.data_ptr(), words)

    def finish(self) -> bool:
        return self.q.block_finish()


class TorchExchange:
    """All-gather of variable-size int32 record buffers over the default process group:
    the sizes first, then the buffers padded to the largest. Under gloo the buffers go
    through host memory; under NCCL they stay on the device."""

    def __init__(self, device="cuda", group=None):
        import torch
        import torch.distributed as dist

        self.torch, self.dist, self.group = torch, dist, group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.host = dist.get_backend(group) == "gloo"
        self.device = torch.device("cpu") if self.host else torch.device(device)

    def allgather(self, records, words: int):
        """[(tensor, words)] of every other rank, in rank order."""
        torch, dist = self.torch, self.dist
        sizes = [torch.zeros(1, dtype=torch.int64, device=self.device) for _ in range(self.world)]
        dist.all_gather(sizes, torch.tensor([words], dtype=torch.int64, device=self.device), group=self.group)
        sizes = [int(s.item()) for s in sizes]
        top = max(sizes)
        if top == 0:
            return []
        mine = torch.zeros(top, dtype=torch.int32, device=self.device)
        if words:
            mine[:words].copy_(records[:words])
        recv = [torch.empty(top, dtype=torch.int32, device=self.device) for _ in range(self.world)]
        dist.all_gather(recv, mine, group=self.group)
        return [(recv[r], sizes[r]) for r in range(self.world) if r != self.rank and sizes[r]]


def solve_sharded(block, exchange, max_executions: int | None = None) -> int:
    """Runs the sharded loop to the fixpoint; returns the loop executions (the last one added
    nothing, as Section 4.3 counts k). Every rank calls it with its own block."""
    block.start()
    k = 0
    while True:
        block.products()
        records, words = block.export()
        for other, w in exchange.allgather(records, words):
            block.import_(other, w)
        k += 1
        if not block.finish():
            return k
        if max_executions is not None and k >= max_executions:
            raise RuntimeError("sharded loop did not converge")


def solve_local(blocks) -> int:
    """All blocks of one solve driven from one process (each block on its own device, or
    several on one): the same loop with the exchange done by copying records between the
    blocks. Returns the loop executions."""
    for b in blocks:
        b.start()
    k = 0
    while True:
        for b in blocks:
            b.products()
        outs = [b.export() for b in blocks]
        for j, b in enumerate(blocks):
            for i, (rec, w) in enumerate(outs):
                if i != j:
                    b.import_(rec, w)
        k += 1
        go = [b.finish() for b in blocks]
        if len(set(go)) != 1:
            raise RuntimeError("row blocks disagree on whether the loop goes on")
        if not go[0]:
            return k
