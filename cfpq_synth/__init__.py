"""Seeded synthetic inputs for context-free path querying (CFPQ).

This module only *draws* inputs: edge-labelled graphs and grammar texts. It holds
none of the closure arithmetic, so both the CPU oracle and the CUDA engine can take
their inputs from here without sharing any part of the method.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014; the 64-bit
finaliser as published by Vigna), evaluated at explicit counters so that every draw
is reproducible independently of vectorisation:

    key(seed, stream) = mix(mix(seed + G) ^ stream)
    u64(key, i)       = mix(key + (i + 1) * G)            G = 0x9E3779B97F4A7C15
    uniform_int(key, i, m) = min(floor((u64 >> 11) * 2**-53 * m), m - 1)

Workload shapes follow the paper's evaluation (Section 6): RDF-like class
hierarchies with subClassOf / type labels where each triple also contributes its
reversed edge with the inverse label, and the same-generation grammars of Query 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def key(seed: int, stream: int) -> np.uint64:
    """Stream key for (seed, stream); independent streams for independent draws."""
    with np.errstate(over="ignore"):
        k = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _G)
    return _mix(k ^ np.uint64(stream & 0xFFFFFFFFFFFFFFFF))


def u64(k, idx) -> np.ndarray:
    """SplitMix64 output number idx (0-based) of stream key k; idx may be an array."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(k) + (idx + np.uint64(1)) * _G)


def uniform01(k, idx) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (u64(k, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_int(k, idx, m) -> np.ndarray:
    """Integers in [0, m) (m may be an array broadcast against idx)."""
    m = np.asarray(m, dtype=np.float64)
    v = np.floor(uniform01(k, idx) * m).astype(np.int64)
    return np.minimum(v, np.asarray(m, dtype=np.int64) - 1)


# --------------------------------------------------------------------------------------
# Graphs
# --------------------------------------------------------------------------------------

@dataclass
class Graph:
    """Edge-labelled directed graph D = (V, E) with V = {0..n-1} (Section 2).

    ``edges`` is an (E, 3) int64 array of (src, label, dst); ``labels`` names the label
    ids. Duplicate edges may occur; they denote the same element of E."""

    n: int
    edges: np.ndarray
    labels: list[str]
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.edges.shape[0])


HIERARCHY_LABELS = ["sc", "sc_r", "ty", "ty_r"]


def hierarchy(n: int, n_classes: int, seed: int = 0, ty_min: int = 1, ty_max: int = 3) -> Graph:
    """RDF-like class hierarchy (shape of the paper's ontologies, Section 6).

    Nodes 0..C-1 are classes, C..n-1 instances. Class c >= 1 has one subClassOf edge
    c -sc-> p with p uniform in [0, c) (class 0 is the root). Instance v has k edges
    v -ty-> c, k uniform in [ty_min, ty_max], each c uniform in [0, C) (drawn with
    replacement, so duplicates may occur). Every edge (o, x, s) is accompanied by
    (s, x_r, o), as the paper does when it converts RDF triples to graphs.
    """
    if not (1 <= n_classes <= n):
        raise ValueError("need 1 <= n_classes <= n")
    C = int(n_classes)
    k_par, k_cnt, k_tgt = key(seed, 1), key(seed, 2), key(seed, 3)
    cls = np.arange(1, C, dtype=np.int64)
    parent = uniform_int(k_par, cls, cls)
    inst = np.arange(C, n, dtype=np.int64)
    span = ty_max - ty_min + 1
    cnt = ty_min + uniform_int(k_cnt, inst, span)
    rep_inst = np.repeat(inst, cnt)
    # slot t of instance v uses counter v * ty_max + t
    slot = np.arange(rep_inst.size, dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    tgt = uniform_int(k_tgt, rep_inst * ty_max + slot, C)
    SC, SCR, TY, TYR = 0, 1, 2, 3
    parts = [
        np.stack([cls, np.full_like(cls, SC), parent], axis=1),
        np.stack([parent, np.full_like(cls, SCR), cls], axis=1),
        np.stack([rep_inst, np.full_like(rep_inst, TY), tgt], axis=1),
        np.stack([tgt, np.full_like(rep_inst, TYR), rep_inst], axis=1),
    ]
    edges = np.concatenate(parts, axis=0).astype(np.int64)
    return Graph(n=n, edges=edges, labels=list(HIERARCHY_LABELS),
                 meta={"kind": "hierarchy", "n_classes": C, "seed": seed})


def two_cycles(p: int, q: int) -> Graph:
    """Two directed cycles sharing node 0: an a-cycle 0->1->..->p-1->0 and a b-cycle
    0->p->p+1->..->p+q-2->0 (q nodes). n = p + q - 1. Labels: a = 0, b = 1."""
    if p < 1 or q < 1:
        raise ValueError("cycle lengths must be >= 1")
    n = p + q - 1
    a_src = np.arange(p, dtype=np.int64)
    a_dst = (a_src + 1) % p
    bnodes = np.concatenate([[0], np.arange(p, p + q - 1)]).astype(np.int64)
    b_src = bnodes
    b_dst = np.roll(bnodes, -1)
    edges = np.concatenate([
        np.stack([a_src, np.zeros_like(a_src), a_dst], axis=1),
        np.stack([b_src, np.ones_like(b_src), b_dst], axis=1)], axis=0)
    return Graph(n=n, edges=edges, labels=["a", "b"], meta={"kind": "two_cycles", "p": p, "q": q})


def random_graph(n: int, n_edges: int, n_labels: int, seed: int = 0) -> Graph:
    """Uniform random multigraph: src, dst in [0, n), label in [0, n_labels)."""
    k = key(seed, 11)
    i = np.arange(n_edges, dtype=np.int64)
    src = uniform_int(k, 3 * i, n)
    lab = uniform_int(k, 3 * i + 1, n_labels)
    dst = uniform_int(k, 3 * i + 2, n)
    edges = np.stack([src, lab, dst], axis=1).astype(np.int64)
    return Graph(n=n, edges=edges, labels=[f"t{j}" for j in range(n_labels)],
                 meta={"kind": "random", "seed": seed})


def communities(n: int, k: int, degree: int = 2, seed: int = 0) -> Graph:
    """k communities of about n / k consecutive nodes each (node v is in community
    v * k // n); every node has `degree` out-edges, label t0, to uniform nodes of its own
    community (drawn with replacement). The transitive closure S -> S S | t0 is dense inside
    each community and empty between them: a closure whose matrices are block-diagonal."""
    kk = key(seed, 13)
    v = np.repeat(np.arange(n, dtype=np.int64), degree)
    c = v * k // n
    lo = (c * n + k - 1) // k           # first node of each community
    hi = ((c + 1) * n + k - 1) // k     # one past its last node
    i = np.arange(v.size, dtype=np.int64)
    dst = lo + uniform_int(kk, i, hi - lo)
    edges = np.stack([v, np.zeros_like(v), dst], axis=1)
    return Graph(n=n, edges=edges, labels=["t0"], meta={"kind": "communities", "k": k, "seed": seed})


# --------------------------------------------------------------------------------------
# Grammars (text form: one production per line, "A B C", "A x" or "A eps"; a symbol is
# a non-terminal iff it appears on some left-hand side; '#' starts a comment)
# --------------------------------------------------------------------------------------

#: Query 1 (Section 6), in the shape of the worked example's normal form with the
#: terminals written directly into the binary rules.
GRAMMAR_Q1 = """\
S sc_r X
S ty_r Y
S sc_r SC
S ty_r TY
X S SC
Y S TY
SC sc
TY ty
"""

#: Same-generation query over subClassOf only: S -> sc_r S sc | sc_r sc.
GRAMMAR_QSC = """\
S sc_r X
S sc_r SC
X S SC
SC sc
"""

#: S -> a S b | a b in normal form.
# The same-generation query read with the opposite subClassOf direction (walk up k sc edges,
# then down k): on these hierarchies R_S holds every pair of classes at the same depth below
# the root, a far denser result than the sc-only query (which only returns the diagonal of
# classes with a child). S -> sc S sc_r | sc sc_r with preterminals.
GRAMMAR_SG = """\
S SC X
S SC SCR
X S SCR
SC sc
SCR sc_r
"""

GRAMMAR_C3 = """\
S A S1
S A B
S1 S B
A a
B b
"""

#: The paper's worked example (Section 4.3), normal form G' exactly as printed.
GRAMMAR_WORKED = """\
S S1 S5
S S3 S6
S S1 S2
S S3 S4
S5 S S2
S6 S S4
S1 sc_r
S2 sc
S3 ty_r
S4 ty
"""

#: The paper's Query 2 (Section 6): S -> B sc | sc ; B -> sc_r B sc | sc_r sc.
GRAMMAR_Q2 = """\
S B sc
S sc
B sc_r B1
B sc_r SC
B1 B SC
SC sc
"""


def worked_example_graph() -> Graph:
    """The 3-node graph of Section 4.3. Its figure is not in the source text; the edges
    are read off the initial matrix T0 (each preterminal derives one terminal)."""
    lab = {x: i for i, x in enumerate(HIERARCHY_LABELS)}
    e = [(0, lab["sc_r"], 0), (0, lab["ty_r"], 1), (1, lab["ty_r"], 2),
         (2, lab["sc"], 0), (2, lab["ty"], 2)]
    return Graph(n=3, edges=np.array(e, dtype=np.int64), labels=list(HIERARCHY_LABELS),
                 meta={"kind": "worked_example"})


def random_grammar_text(n_nt: int, n_terms: int, n_binary: int, n_unary: int,
                        n_eps: int, seed: int = 0) -> str:
    """A random grammar in (weak) normal form over terminals t0..t{n_terms-1}.

    Every non-terminal N0..N{n_nt-1} gets at least one unary production so that each
    is a left-hand side."""
    k = key(seed, 21)
    lines = []
    c = 0
    for a in range(n_nt):
        t = int(uniform_int(k, c, n_terms)); c += 1
        lines.append(f"N{a} t{t}")
    for _ in range(max(0, n_unary - n_nt)):
        a = int(uniform_int(k, c, n_nt)); t = int(uniform_int(k, c + 1, n_terms)); c += 2
        lines.append(f"N{a} t{t}")
    for _ in range(n_binary):
        a, b, d = (int(x) for x in uniform_int(k, np.arange(c, c + 3), n_nt)); c += 3
        lines.append(f"N{a} N{b} N{d}")
    for _ in range(n_eps):
        a = int(uniform_int(k, c, n_nt)); c += 1
        lines.append(f"N{a} eps")
    return "\n".join(lines) + "\n"


# --------------------------------------------------------------------------------------
# Workloads of the benchmark configurations
# --------------------------------------------------------------------------------------

def batch_queries(count: int = 256, n_lo: int = 64, n_hi: int = 4096, class_frac: float = 0.3,
                  seed: int = 0):
    """Independent queries: n log-uniform in [n_lo, n_hi], hierarchy graph with
    C = max(1, round(class_frac * n)) classes, grammar Q1 or QSC chosen uniformly.

    Returns a list of (Graph, grammar_text)."""
    k = key(seed, 31)
    out = []
    for q in range(count):
        u = float(uniform01(k, 2 * q))
        n = int(math.floor(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
        n = max(n_lo, min(n, n_hi))
        C = max(1, int(round(class_frac * n)))
        g = hierarchy(n, C, seed=seed * 100003 + q)
        gram = GRAMMAR_Q1 if int(uniform_int(k, 2 * q + 1, 2)) == 0 else GRAMMAR_QSC
        out.append((g, gram))
    return out


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    k = key(seed, 41)
    u = uniform01(k, np.arange(count))
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)
