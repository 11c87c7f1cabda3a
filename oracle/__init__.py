"""CPU oracle for relational-semantics context-free path querying (CFPQ).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product path never does.

Contents, each written from the paper and checked by the pins in ``tests/``:

* ``parse_grammar``  -- reads grammar text into the normal form of Section 2 (rules
  A -> B C, A -> x, plus A -> eps), introducing one preterminal per terminal that
  occurs inside a binary production, as the paper does when it rewrites the
  same-generation grammar into G' (Section 4.3).
* ``hellings``       -- the relations R_A of Section 2 by the worklist algorithm in
  ``cfpq_oracle.c`` (plain C, exact).
* ``matrix_closure`` -- Algorithm 1 (Section 4.2) written literally over |N| Boolean
  matrices: T <- T u (T x T) with the subset product of Section 2, until T stops
  changing; returns every intermediate T_k and the loop count k of Section 4.3.
* ``brute_force``    -- enumerates walks up to a length bound and runs CYK on their
  label strings (tiny inputs only).
* ``check_*``        -- properties any correct result has (Theorem 2 / Section 4.2):
  seed inclusion, closure under every production, witnesses for derived pairs.

Naming convention shared with the engine's grammar reader (an interface, not
arithmetic): non-terminals are numbered in order of first appearance as a left-hand
side, then preterminals in order of first appearance inside binary productions; the
preterminal of terminal ``x`` is named ``<x>``; terminal ids are positions in the
graph's label list.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import build as _build


# --------------------------------------------------------------------------------------
# Grammar text -> normal form (Section 2; preterminals as in Section 4.3)
# --------------------------------------------------------------------------------------

@dataclass
class CNF:
    names: list            # non-terminal names, id = position
    unary: list            # (A, terminal id)
    binary: list           # (A, B, C)
    eps: list              # A with A -> eps
    labels: list           # terminal names, id = position

    def id(self, name: str) -> int:
        return self.names.index(name)


def parse_grammar(text: str, labels) -> CNF:
    rows = []
    for ln in text.splitlines():
        ln = ln.split("#", 1)[0].strip()
        if not ln:
            continue
        toks = ln.split()
        if len(toks) not in (2, 3):
            raise ValueError(f"bad production: {ln!r}")
        for t in toks:
            if "<" in t or ">" in t:
                raise ValueError(f"symbol may not contain '<' or '>': {t!r}")
        rows.append(toks)
    names = []
    for toks in rows:
        if toks[0] == "eps":
            raise ValueError("'eps' cannot be a left-hand side")
        if toks[0] not in names:
            names.append(toks[0])
    lab = {x: i for i, x in enumerate(labels)}
    nts = set(names)
    unary, binary, eps = [], [], []
    pre = {}

    def operand(sym):
        if sym in nts:
            return names.index(sym)
        if sym not in lab:
            raise ValueError(f"unknown terminal {sym!r}")
        if sym not in pre:
            pre[sym] = None
        return ("pre", sym)

    pending = []
    for toks in rows:
        a = names.index(toks[0])
        if len(toks) == 2:
            s = toks[1]
            if s == "eps":
                eps.append(a)
            elif s in nts:
                raise ValueError(f"chain production {toks[0]} -> {s} is not in normal form")
            elif s in lab:
                unary.append((a, lab[s]))
            else:
                raise ValueError(f"unknown terminal {s!r}")
        else:
            if "eps" in toks[1:]:
                raise ValueError("eps inside a binary production")
            pending.append((a, operand(toks[1]), operand(toks[2])))
    for sym in pre:
        pre[sym] = len(names)
        names.append(f"<{sym}>")
        unary.append((pre[sym], lab[sym]))

    def res(x):
        return pre[x[1]] if isinstance(x, tuple) else x

    for a, b, c in pending:
        binary.append((a, res(b), res(c)))
    return CNF(names=names, unary=unary, binary=binary, eps=eps, labels=list(labels))


# --------------------------------------------------------------------------------------
# Hellings-style worklist (C)
# --------------------------------------------------------------------------------------

_libs = {}


def _lib(plant: int = 0):
    if plant not in _libs:
        lib = ctypes.CDLL(_build.build(plant))
        P = ctypes.POINTER
        i32p, i64p, u32p = P(ctypes.c_int32), P(ctypes.c_int64), P(ctypes.c_uint32)
        lib.oracle_solve.restype = ctypes.c_void_p
        lib.oracle_solve.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     i32p, ctypes.c_int32, i32p, ctypes.c_int32,
                                     i32p, ctypes.c_int32, i64p, ctypes.c_int64]
        lib.oracle_count.restype = ctypes.c_int64
        lib.oracle_count.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        lib.oracle_pops.restype = ctypes.c_int64
        lib.oracle_pops.argtypes = [ctypes.c_void_p]
        lib.oracle_copy.restype = ctypes.c_int64
        lib.oracle_copy.argtypes = [ctypes.c_void_p, ctypes.c_int32, u32p, ctypes.c_int64]
        lib.oracle_has.restype = ctypes.c_int
        lib.oracle_has.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_release.restype = None
        lib.oracle_release.argtypes = [ctypes.c_void_p]
        _libs[plant] = lib
    return _libs[plant]


def _arr(x, dtype):
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype).reshape(-1))
    if a.size == 0:
        a = np.zeros(1, dtype=dtype)
    return a


class HellingsResult:
    """R_A for every non-terminal, kept in the C oracle's bitsets."""

    def __init__(self, cnf: CNF, n: int, edges, plant: int = 0):
        self.cnf, self.n = cnf, n
        self._lib = _lib(plant)
        P = ctypes.POINTER
        un = _arr(cnf.unary, np.int32)
        bi = _arr(cnf.binary, np.int32)
        ep = _arr(cnf.eps, np.int32)
        ed = _arr(edges, np.int64)
        self._keep = (un, bi, ep, ed)
        self._h = self._lib.oracle_solve(
            len(cnf.names), len(cnf.labels), n,
            un.ctypes.data_as(P(ctypes.c_int32)), len(cnf.unary),
            bi.ctypes.data_as(P(ctypes.c_int32)), len(cnf.binary),
            ep.ctypes.data_as(P(ctypes.c_int32)), len(cnf.eps),
            ed.ctypes.data_as(P(ctypes.c_int64)), int(np.asarray(edges).reshape(-1, 3).shape[0]))
        if not self._h:
            raise ValueError("oracle rejected the input (id out of range) or ran out of memory")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_release(h)
            self._h = None

    def count(self, A) -> int:
        a = self.cnf.id(A) if isinstance(A, str) else A
        return int(self._lib.oracle_count(self._h, a))

    def pairs(self, A) -> np.ndarray:
        """R_A as a sorted (k, 2) uint32 array of (m, n)."""
        a = self.cnf.id(A) if isinstance(A, str) else A
        k = self.count(a)
        buf = np.zeros((max(k, 1), 2), dtype=np.uint32)
        got = self._lib.oracle_copy(self._h, a, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), k)
        assert got == k
        return buf[:k]

    def has(self, A, m: int, n: int) -> bool:
        a = self.cnf.id(A) if isinstance(A, str) else A
        return bool(self._lib.oracle_has(self._h, a, m, n))

    @property
    def pops(self) -> int:
        return int(self._lib.oracle_pops(self._h))

    def as_sets(self) -> dict:
        return {nm: set(map(tuple, self.pairs(i).tolist())) for i, nm in enumerate(self.cnf.names)}


def hellings(graph, grammar_text: str, plant: int = 0) -> HellingsResult:
    cnf = parse_grammar(grammar_text, graph.labels)
    return HellingsResult(cnf, graph.n, graph.edges, plant=plant)


# --------------------------------------------------------------------------------------
# Algorithm 1, literally (Section 4.2): Boolean matrices, Jacobi update
# --------------------------------------------------------------------------------------

def initial_matrices(cnf: CNF, n: int, edges) -> dict:
    """Matrix initialisation of Algorithm 1: T_ij gets {A | A -> x} for every edge
    (i, x, j); multiple edges add the union of their heads. A -> eps adds A on the
    diagonal (the empty walk from m to m)."""
    T = {a: np.zeros((n, n), dtype=bool) for a in range(len(cnf.names))}
    heads = {}
    for a, t in cnf.unary:
        heads.setdefault(t, []).append(a)
    for src, lab, dst in np.asarray(edges, dtype=np.int64).reshape(-1, 3):
        for a in heads.get(int(lab), []):
            T[a][src, dst] = True
    for a in cnf.eps:
        np.fill_diagonal(T[a], True)
    return T


def matrix_product(cnf: CNF, T: dict) -> dict:
    """(T x T)_ij = union over k of T_ik . T_kj with N1 . N2 = {A | A -> B C, B in N1,
    C in N2} (Section 2), computed as one Boolean matrix product per production."""
    n = next(iter(T.values())).shape[0]
    P = {a: np.zeros((n, n), dtype=bool) for a in T}
    for a, b, c in cnf.binary:
        P[a] |= (T[b].astype(np.int64) @ T[c].astype(np.int64)) > 0
    return P


def matrix_closure(graph, grammar_text: str, max_iter: int | None = None):
    """Runs Algorithm 1 and returns (cnf, snapshots, k): snapshots[i] = T_i (T_0 the
    initial matrix), k = number of loop executions, the last one being the execution
    that left T unchanged (k = 6 for the worked example of Section 4.3)."""
    cnf = parse_grammar(grammar_text, graph.labels)
    T = initial_matrices(cnf, graph.n, graph.edges)
    snaps = [{a: m.copy() for a, m in T.items()}]
    k = 0
    while True:
        k += 1
        P = matrix_product(cnf, T)
        new = {a: T[a] | P[a] for a in T}
        changed = any((new[a] != T[a]).any() for a in T)
        T = new
        if not changed:
            break
        snaps.append({a: m.copy() for a, m in T.items()})
        if max_iter is not None and k >= max_iter:
            break
    return cnf, snaps, k


def single_path_lengths(graph, grammar_text: str, max_iter: int | None = None, _plant: str | None = None):
    """The closure of Section 5 (single-path semantics): every pair carries the length of
    one path whose labels the non-terminal derives. a^(1): (A, 1) for every edge (i, x, j)
    with A -> x (and, reading A -> eps as the empty walk, (A, 0) on the diagonal); each loop
    execution p adds (A, l_B + l_C) at (i, j) for A -> B C, (B, l_B) in a^(p-1)_{i,k} and
    (C, l_C) in a^(p-1)_{k,j}, but only where A is not at (i, j) yet: the length first found
    is kept. Where one execution finds several lengths for the same new (A, i, j) the paper
    does not say which is kept; this reading keeps the smallest (so the result is unique).
    Returns (cnf, lengths, k): lengths[A] = {(i, j): l}, k the loop count as in
    ``matrix_closure``. Plain dictionaries; small inputs only. ``_plant`` (tests only) puts a
    known mistake in: "plus_one" (l_B + l_C + 1), "last_wins" (a later length replaces the
    first), "max_tie" (the largest of one execution's lengths)."""
    cnf = parse_grammar(grammar_text, graph.labels)
    n = graph.n
    L = {a: {} for a in range(len(cnf.names))}
    heads = {}
    for a, t in cnf.unary:
        heads.setdefault(t, []).append(a)
    for src, lab, dst in np.asarray(graph.edges, dtype=np.int64).reshape(-1, 3):
        for a in heads.get(int(lab), []):
            L[a][(int(src), int(dst))] = 1
    for a in cnf.eps:
        for m in range(n):
            L[a][(m, m)] = 0
    # right operands by row, for the joins
    k = 0
    while True:
        k += 1
        by_row = {a: {} for a in L}
        for a, pairs in L.items():
            for (i, j), l in pairs.items():
                by_row[a].setdefault(i, []).append((j, l))
        found = {}
        for a, b, c in cnf.binary:
            for (i, kk), lb in L[b].items():
                for j, lc in by_row[c].get(kk, []):
                    if (i, j) in L[a] and _plant != "last_wins":
                        continue
                    key = (a, i, j)
                    cand = lb + lc + (1 if _plant == "plus_one" else 0)
                    if _plant == "last_wins" and (i, j) in L[a] and L[a][(i, j)] == cand:
                        continue
                    better = cand > found[key] if _plant == "max_tie" and key in found else \
                        (key not in found or cand < found[key])
                    if better:
                        found[key] = cand
        for (a, i, j), l in found.items():
            L[a][(i, j)] = l
        if not found:
            break
        if max_iter is not None and k >= max_iter:
            break
    return cnf, L, k


def walk_exists(graph, cnf, a: int, i: int, j: int, length: int) -> bool:
    """Brute force: is there a walk of exactly `length` edges from i to j whose label string
    non-terminal a derives (CYK on every walk label)? Tiny inputs only."""
    by_src = {}
    for src, lab, dst in np.asarray(graph.edges, dtype=np.int64).reshape(-1, 3):
        by_src.setdefault(int(src), []).append((int(lab), int(dst)))
    if length == 0:
        return i == j and a in cyk_table(cnf, [])[0][0]  # the nullable non-terminals
    frontier = {(i, ())}
    for _ in range(length):
        nxt = set()
        for node, labels in frontier:
            for lab, dst in by_src.get(node, []):
                nxt.add((dst, labels + (lab,)))
        frontier = nxt
    for node, labels in frontier:
        if node == j and a in cyk_table(cnf, list(labels))[0][length]:
            return True
    return False


def matrix_closure_sparse(graph, grammar_text: str, max_iter: int | None = None):
    """Algorithm 1 as in ``matrix_closure`` but with sparse Boolean matrices (scipy CSR
    products as the library primitive, the representation of the paper's sCPU variant),
    for sizes where dense n x n products are too slow. Returns (cnf, T, k) with T the
    final matrices and k the loop count."""
    import scipy.sparse as sp

    cnf = parse_grammar(grammar_text, graph.labels)
    n = graph.n
    heads = {}
    for a, t in cnf.unary:
        heads.setdefault(t, []).append(a)
    rows = {a: [] for a in range(len(cnf.names))}
    cols = {a: [] for a in range(len(cnf.names))}
    for src, lab, dst in np.asarray(graph.edges, dtype=np.int64).reshape(-1, 3):
        for a in heads.get(int(lab), []):
            rows[a].append(int(src))
            cols[a].append(int(dst))
    for a in cnf.eps:
        rows[a].extend(range(n))
        cols[a].extend(range(n))

    def mat(r, c):
        m = sp.csr_matrix((np.ones(len(r), dtype=np.int64), (np.asarray(r, dtype=np.int64),
                                                              np.asarray(c, dtype=np.int64))), shape=(n, n))
        m.data[:] = 1
        return m

    T = {a: mat(rows[a], cols[a]) for a in rows}
    k = 0
    while True:
        k += 1
        new = {a: T[a].copy() for a in T}
        for a, b, c in cnf.binary:
            new[a] = new[a] + (T[b] @ T[c])
        changed = False
        for a in T:
            new[a].data[:] = 1
            new[a].eliminate_zeros()
            if new[a].nnz != T[a].nnz:
                changed = True
        T = new
        if not changed or (max_iter is not None and k >= max_iter):
            break
    return cnf, T, k


# --------------------------------------------------------------------------------------
# Brute force: walks + CYK (tiny inputs)
# --------------------------------------------------------------------------------------

def cyk_table(cnf: CNF, word) -> list:
    """CYK over a terminal-id string, extended to productions A -> eps: cell (i, j)
    holds every non-terminal deriving word[i:j]; empty spans hold the nullable
    non-terminals, and each cell is iterated to a fixpoint because a split may have
    an empty side."""
    L = len(word)
    tab = [[set() for _ in range(L + 1)] for _ in range(L + 1)]
    nullable = set(cnf.eps)
    changed = True
    while changed:
        changed = False
        for a, b, c in cnf.binary:
            if b in nullable and c in nullable and a not in nullable:
                nullable.add(a)
                changed = True
    for i in range(L + 1):
        tab[i][i] = set(nullable)
    for i in range(L):
        for a, t in cnf.unary:
            if t == word[i]:
                tab[i][i + 1].add(a)
    for span in range(1, L + 1):
        for i in range(0, L - span + 1):
            j = i + span
            cell = tab[i][j]
            while True:
                before = len(cell)
                for k in range(i, j + 1):
                    left, right = tab[i][k], tab[k][j]
                    if not left or not right:
                        continue
                    for a, b, c in cnf.binary:
                        if b in left and c in right:
                            cell.add(a)
                if len(cell) == before:
                    break
    return tab


def brute_force(graph, grammar_text: str, max_len: int) -> dict:
    """{name: set of (m, n)} over all walks of length <= max_len (length 0 included):
    (m, n) is in R_A iff some walk m -> n of at most max_len edges has a label string
    that A derives (checked by CYK)."""
    cnf = parse_grammar(grammar_text, graph.labels)
    adj = {}
    for s, l, d in np.asarray(graph.edges, dtype=np.int64).reshape(-1, 3):
        adj.setdefault(int(s), set()).add((int(l), int(d)))
    res = {nm: set() for nm in cnf.names}
    cache = {}
    for start in range(graph.n):
        frontier = [((), start)]
        for length in range(0, max_len + 1):
            nxt = set()
            for word, node in frontier:
                if word not in cache:
                    tab = cyk_table(cnf, list(word))
                    cache[word] = tab[0][len(word)]
                for a in cache[word]:
                    res[cnf.names[a]].add((start, node))
                if length < max_len:
                    for l, d in adj.get(node, ()):
                        nxt.add((word + (l,), d))
            frontier = sorted(nxt)
    return res


# --------------------------------------------------------------------------------------
# Properties that hold for any correct result (used at sizes the oracle cannot run)
# --------------------------------------------------------------------------------------

def _to_sparse(pairs, n):
    import scipy.sparse as sp
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    return sp.csr_matrix((np.ones(p.shape[0], dtype=np.int64), (p[:, 0], p[:, 1])), shape=(n, n))


def check_seed_included(cnf: CNF, n: int, edges, result: dict) -> bool:
    """Every seeded pair (edge with a unary head, eps diagonal) is in the result."""
    heads = {}
    for a, t in cnf.unary:
        heads.setdefault(t, []).append(a)
    sets = {a: _to_sparse(result[nm], n) for a, nm in enumerate(cnf.names)}
    for src, lab, dst in np.asarray(edges, dtype=np.int64).reshape(-1, 3):
        for a in heads.get(int(lab), []):
            if sets[a][src, dst] == 0:
                return False
    for a in cnf.eps:
        if (sets[a].diagonal() == 0).any():
            return False
    return True


def check_closed(cnf: CNF, n: int, result: dict) -> bool:
    """One more application of T <- T u (T x T) adds nothing (the loop's exit test in
    Algorithm 1): for every production A -> B C, R_B R_C is contained in R_A."""
    mats = {a: _to_sparse(result[nm], n) for a, nm in enumerate(cnf.names)}
    for a, b, c in cnf.binary:
        prod = (mats[b] @ mats[c]).tocoo()
        if prod.nnz == 0:
            continue
        have = mats[a][prod.row, prod.col]
        if (np.asarray(have).reshape(-1) == 0).any():
            return False
    return True


def check_witnessed(cnf: CNF, n: int, edges, result: dict, sample=None, seed: int = 0) -> bool:
    """Every pair that is not a seed has a derivation step: some A -> B C and k with
    (m, k) in R_B and (k, n) in R_C (Lemma 3's inductive step). ``sample`` bounds the
    number of pairs checked per non-terminal."""
    mats = {a: _to_sparse(result[nm], n) for a, nm in enumerate(cnf.names)}
    heads = {}
    for a, t in cnf.unary:
        heads.setdefault(t, []).append(a)
    seeds = {a: set() for a in mats}
    for src, lab, dst in np.asarray(edges, dtype=np.int64).reshape(-1, 3):
        for a in heads.get(int(lab), []):
            seeds[a].add((int(src), int(dst)))
    rng = np.random.default_rng(seed)
    for a, nm in enumerate(cnf.names):
        pairs = np.asarray(result[nm], dtype=np.int64).reshape(-1, 2)
        if sample is not None and pairs.shape[0] > sample:
            pairs = pairs[rng.choice(pairs.shape[0], sample, replace=False)]
        for m, nn in pairs.tolist():
            if (m, nn) in seeds[a] or (a in cnf.eps and m == nn):
                continue
            ok = False
            for a2, b, c in cnf.binary:
                if a2 != a:
                    continue
                row_b = mats[b].getrow(m).toarray().reshape(-1) != 0
                col_c = mats[c].getcol(nn).toarray().reshape(-1) != 0
                if (row_b & col_c).any():
                    ok = True
                    break
            if not ok:
                return False
    return True

