"""B300 (sm_103a) engine for relational-semantics context-free path querying.

Thin Python binding over the C ABI in ``include/cfpq.h`` (``libcfpq.so``): argument
marshalling only; every step of the closure runs in the library's CUDA kernels. There is
no CPU fallback: if the library is missing or has no device to run on, calls raise.

    g = Grammar(text, labels)                 # normal form with preterminals (Section 4.3)
    q = Query(g, n, edges)                    # edges: (E, 3) ints (src, label, dst)
    q.solve()                                 # Algorithm 1 on the GPU
    q.get("S")                                # R_S as a sorted (k, 2) uint32 array
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcfpq.so")

OK, ERR_INVALID, ERR_NOMEM, ERR_NOT_SOLVED, ERR_ITER_LIMIT, ERR_TIMEOUT, ERR_CUDA, ERR_BUFFER, \
    ERR_UNSUPPORTED, ERR_NOT_FOUND = range(10)
SCHED_INPLACE, SCHED_JACOBI, SCHED_AUTO = 0, 1, 2
TUNE_CLASSES = 24
PATH_AUTO, PATH_TENSOR, PATH_GATHER, PATH_WORKLIST = 0, 1, 2, 3
TENSOR_AUTO, TENSOR_FP8, TENSOR_FP4 = 0, 1, 2


class CfpqError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {_lib().cfpq_strerror(code).decode()} (status {code})")
        self.code = code


class Rule1(ctypes.Structure):
    _fields_ = [("lhs", ctypes.c_int32), ("term", ctypes.c_int32)]


class Rule2(ctypes.Structure):
    _fields_ = [("lhs", ctypes.c_int32), ("b", ctypes.c_int32), ("c", ctypes.c_int32)]


class GrammarCNF(ctypes.Structure):
    _fields_ = [("n_nonterm", ctypes.c_int32), ("n_term", ctypes.c_int32),
                ("unary", ctypes.POINTER(Rule1)), ("n_unary", ctypes.c_int32),
                ("binary", ctypes.POINTER(Rule2)), ("n_binary", ctypes.c_int32),
                ("eps_lhs", ctypes.POINTER(ctypes.c_int32)), ("n_eps", ctypes.c_int32)]


class Edge(ctypes.Structure):
    _fields_ = [("src", ctypes.c_uint32), ("label", ctypes.c_int32), ("dst", ctypes.c_uint32)]


class Triple(ctypes.Structure):
    _fields_ = [("A", ctypes.c_int32), ("m", ctypes.c_uint32), ("n", ctypes.c_uint32)]


_PINNED = None  # torch, when its CUDA host allocator can stage results (False: plain numpy)
_PINNED_MAX_BYTES = 1 << 30  # larger results go to ordinary memory (pinning gigabytes can fail)


def _host_words(rows: int, cols: int) -> np.ndarray:
    """A (rows, cols) uint32 host array for results copied from the device. Page-locked memory
    from torch's caching host allocator where CUDA is up: the device-to-host copy then runs at
    the link's rate with no staging or page faults, and the block returns to the allocator's
    cache when the array is dropped (the array keeps its tensor alive)."""
    global _PINNED
    if _PINNED is None:
        try:
            import torch

            _PINNED = torch if torch.cuda.is_available() else False
        except ImportError:
            _PINNED = False
    if _PINNED and rows * cols * 4 <= _PINNED_MAX_BYTES:
        try:
            t = _PINNED.empty((rows, cols), dtype=_PINNED.int32, pin_memory=True)
            return t.numpy().view("<u4")
        except RuntimeError:  # page-locked memory exhausted: ordinary memory works as well
            pass
    return np.empty((rows, cols), dtype="<u4")


def _triple_rows(k: int) -> np.ndarray:
    """A host buffer for k cfpq_triple records as a (k, 3) uint32 array: the record is three
    32-bit words, and A (a non-terminal id) and m, n (< CFPQ_MAX_NODES) are non-negative,
    so the unsigned view reads every field exactly."""
    return _host_words(max(k, 1), 3)


def _triple_ptr(buf: np.ndarray):
    return buf.ctypes.data_as(ctypes.POINTER(Triple))


class Options(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("path", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("max_iter", ctypes.c_int64), ("timeout_s", ctypes.c_double),
                ("lengths", ctypes.c_int32), ("dense_tensor", ctypes.c_int32), ("tensor_kind", ctypes.c_int32),
                ("row_begin", ctypes.c_uint32), ("row_end", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("new_bits", ctypes.c_int64), ("seed_bits", ctypes.c_int64),
                ("tensor_products", ctypes.c_int64), ("gather_products", ctypes.c_int64),
                ("dense_ops", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("n_pad", ctypes.c_uint32), ("status", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("product_launches", ctypes.c_int64),
                ("product_ms", ctypes.c_double), ("tensor_ms", ctypes.c_double),
                ("tensor_launches", ctypes.c_int64), ("product_bytes", ctypes.c_double),
                ("worklist_items", ctypes.c_int64), ("schedule", ctypes.c_int32), ("gather_cpl", ctypes.c_int32),
                ("useful_ops", ctypes.c_double), ("lengths_ms", ctypes.c_double),
                ("lengths_launches", ctypes.c_int64), ("lengths_splits", ctypes.c_double),
                ("tensor_live_ops", ctypes.c_double), ("worklist_setup_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerOptions(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("rounds_per_step", ctypes.c_int32),
                ("max_resident", ctypes.c_int32)]


class QueryInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("iterations", ctypes.c_int64),
                ("n_nonterm", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("resident", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("launches", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("budget_bytes", ctypes.c_uint64), ("used_bytes", ctypes.c_uint64),
                ("peak_used_bytes", ctypes.c_uint64), ("admit_ms", ctypes.c_double), ("launch_ms", ctypes.c_double),
                ("retire_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


BATCH_GROUPED, BATCH_ALONE = 0, 1


class BatchTuning(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int32), ("cpl", ctypes.c_int32 * TUNE_CLASSES),
                ("schedule", ctypes.c_int32 * TUNE_CLASSES), ("product", ctypes.c_int32 * TUNE_CLASSES)]

    def as_dict(self):
        """blocks_per_sm plus the non-built-in entries per size class."""
        return {"blocks_per_sm": self.blocks_per_sm,
                "cpl": {c: self.cpl[c] for c in range(TUNE_CLASSES) if self.cpl[c]},
                "schedule": {c: self.schedule[c] for c in range(TUNE_CLASSES) if self.schedule[c]},
                "alone": sorted(c for c in range(TUNE_CLASSES) if self.product[c] == BATCH_ALONE)}


class TensorPeaks(ctypes.Structure):
    _fields_ = [("f8f6f4_tflops", ctypes.c_double), ("mxf4_tflops", ctypes.c_double),
                ("f8f6f4_ops_per_clk_sm", ctypes.c_double), ("mxf4_ops_per_clk_sm", ctypes.c_double),
                ("f8f6f4_exact", ctypes.c_int32), ("mxf4_exact", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneReport(ctypes.Structure):
    _fields_ = [("trials", ctypes.c_int32), ("default_ms", ctypes.c_double), ("best_ms", ctypes.c_double)]


QUERY_QUEUED, QUERY_RUNNING, QUERY_DONE, QUERY_FAILED = range(4)

_LIB = None

_P, _VP = ctypes.POINTER, ctypes.c_void_p
#: signature of every function ``include/cfpq.h`` declares
SIGNATURES = {
    "cfpq_options_default": (ctypes.c_int, [_P(Options)]),
    "cfpq_create": (ctypes.c_int, [_P(GrammarCNF), ctypes.c_uint32, _P(Edge), ctypes.c_size_t, _P(Options),
                                   _P(_VP)]),
    "cfpq_solve": (ctypes.c_int, [_VP, _VP]),
    "cfpq_get": (ctypes.c_int, [_VP, ctypes.c_int32, _P(Triple), ctypes.c_size_t, _P(ctypes.c_size_t)]),
    "cfpq_get_all": (ctypes.c_int, [_VP, _P(Triple), ctypes.c_size_t, _P(ctypes.c_size_t)]),
    "cfpq_get_device": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_size_t, _P(ctypes.c_size_t)]),
    "cfpq_get_all_device": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t, _P(ctypes.c_size_t)]),
    "cfpq_count": (ctypes.c_int, [_VP, ctypes.c_int32, _P(ctypes.c_size_t)]),
    "cfpq_get_lengths": (ctypes.c_int, [_VP, ctypes.c_int32, _P(Triple), _P(ctypes.c_uint32), ctypes.c_size_t,
                                        _P(ctypes.c_size_t)]),
    "cfpq_get_path": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32, _P(ctypes.c_uint32),
                                     _P(ctypes.c_int32), ctypes.c_size_t, _P(ctypes.c_size_t)]),
    "cfpq_stats_get": (ctypes.c_int, [_VP, _P(Stats)]),
    "cfpq_destroy": (None, [_VP]),
    "cfpq_trim_memory": (ctypes.c_int, [ctypes.c_size_t]),
    "cfpq_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "cfpq_grammar_parse": (ctypes.c_int, [ctypes.c_char_p, _P(ctypes.c_char_p), ctypes.c_int32, _P(_VP),
                                          ctypes.c_char_p, ctypes.c_size_t]),
    "cfpq_grammar_cnf_of": (_P(GrammarCNF), [_VP]),
    "cfpq_grammar_name": (ctypes.c_char_p, [_VP, ctypes.c_int32]),
    "cfpq_grammar_free": (None, [_VP]),
    "cfpq_solve_batch": (ctypes.c_int, [_P(_VP), ctypes.c_int32, _VP]),
    "cfpq_batch_tuning_default": (None, [_P(BatchTuning)]),
    "cfpq_batch_tuning_get": (ctypes.c_int, [_P(BatchTuning)]),
    "cfpq_batch_tuning_set": (ctypes.c_int, [_P(BatchTuning)]),
    "cfpq_autotune_batch": (ctypes.c_int, [_P(_VP), ctypes.c_int32, _VP, _P(BatchTuning), _P(TuneReport)]),
    "cfpq_solve_batch_tuned": (ctypes.c_int, [_P(_VP), ctypes.c_int32, _P(BatchTuning), _VP]),
    "cfpq_measure_mma_sync_peaks": (ctypes.c_int, [_P(ctypes.c_double), _P(ctypes.c_double)]),
    "cfpq_measure_tensor_peaks": (ctypes.c_int, [_VP]),
    "cfpq_batch_last_profile": (ctypes.c_int, [_P(ctypes.c_double), ctypes.c_int32, _P(ctypes.c_int64),
                                               _P(ctypes.c_double), ctypes.c_int32]),
    "cfpq_server_options_default": (ctypes.c_int, [_P(ServerOptions)]),
    "cfpq_server_create": (ctypes.c_int, [_P(ServerOptions), _P(_VP)]),
    "cfpq_server_submit": (ctypes.c_int, [_VP, _P(GrammarCNF), ctypes.c_uint32, _P(Edge), ctypes.c_size_t,
                                          ctypes.c_int32, _P(ctypes.c_int64)]),
    "cfpq_server_step": (ctypes.c_int, [_VP, _P(ctypes.c_int32)]),
    "cfpq_server_completed": (ctypes.c_int, [_VP, _P(ctypes.c_int64), ctypes.c_size_t, _P(ctypes.c_size_t)]),
    "cfpq_server_query_info": (ctypes.c_int, [_VP, ctypes.c_int64, _P(QueryInfo)]),
    "cfpq_server_result": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int32, _P(Triple), ctypes.c_size_t,
                                          _P(ctypes.c_size_t)]),
    "cfpq_server_release": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "cfpq_server_stats_get": (ctypes.c_int, [_VP, _P(ServerStats)]),
    "cfpq_server_destroy": (None, [_VP]),
    "cfpq_extract_pairs_noalloc": (ctypes.c_int, [_VP, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                  ctypes.c_int32, _VP, ctypes.c_size_t, _P(ctypes.c_size_t), _VP]),
    "cfpq_block_start": (ctypes.c_int, [_VP, _VP]),
    "cfpq_block_products": (ctypes.c_int, [_VP, _VP]),
    "cfpq_block_export": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t, _P(ctypes.c_size_t), _VP]),
    "cfpq_block_import": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t, _VP]),
    "cfpq_block_finish": (ctypes.c_int, [_VP, _VP, _P(ctypes.c_int32)]),
    "cfpq_state_size": (ctypes.c_int, [_VP, _P(ctypes.c_size_t)]),
    "cfpq_export_state": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "cfpq_import_state": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "cfpq_resume": (ctypes.c_int, [_VP, _VP, ctypes.c_int64]),
}
EXPORTS = sorted(SIGNATURES)


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA engine library not built: {LIB_PATH} "
                               "(run `python -m paper_1707_01007_b300.build`)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        _LIB = lib
    return _LIB


def library():
    """The loaded ``libcfpq.so`` (ctypes handle)."""
    return _lib()


def _check(code, what):
    if code != OK:
        raise CfpqError(code, what)


class Grammar:
    """A grammar read by the library's own reader (``cfpq_grammar_parse``)."""

    def __init__(self, text: str, labels):
        self.labels = list(labels)
        arr = (ctypes.c_char_p * max(1, len(self.labels)))(*[s.encode() for s in self.labels])
        h = ctypes.c_void_p()
        err = ctypes.create_string_buffer(256)
        code = _lib().cfpq_grammar_parse(text.encode(), arr, len(self.labels), ctypes.byref(h), err, 256)
        if code != OK:
            raise ValueError(f"grammar rejected: {err.value.decode()}")
        self._h = h
        self.cnf = _lib().cfpq_grammar_cnf_of(h)
        self.names = [_lib().cfpq_grammar_name(h, i).decode() for i in range(self.cnf.contents.n_nonterm)]

    def id(self, name: str) -> int:
        return self.names.index(name)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _LIB is not None:
            _LIB.cfpq_grammar_free(h)
            self._h = None


_EDGE_DTYPE = np.dtype([("src", "<u4"), ("label", "<i4"), ("dst", "<u4")])


def _edges_struct(edges):
    """The edges as cfpq_edge records, in page-locked memory where CUDA is up (the library's
    upload from it is a direct copy; see _host_words)."""
    e = np.asarray(edges).reshape(-1, 3)
    if e.size and int(e.max()) >= 1 << 32:  # would wrap into the 32-bit fields (the library checks the rest)
        raise CfpqError(ERR_INVALID, "edge field out of range")
    words = _host_words(e.shape[0], 3)
    np.copyto(words, e, casting="unsafe")  # one pass; a negative label keeps its int32 bits
    return words.view(_EDGE_DTYPE).reshape(-1)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(int(stream.cuda_stream))  # torch.cuda.Stream


class Query:
    """One CFPQ query (graph + grammar) resident on the device (``cfpq_create``)."""

    def __init__(self, grammar: Grammar, n: int, edges, schedule: int = SCHED_INPLACE, path: int = PATH_AUTO,
                 use_graph: bool = True, max_iter: int = 0, timeout_s: float = 0.0, profile: bool = False,
                 lengths: bool = False, dense_tensor: bool = False, tensor_kind: int = TENSOR_AUTO,
                 row_begin: int = 0, row_end: int = 0):
        self.grammar = grammar
        self.n = int(n)
        self._h = None
        opt = Options()
        _lib().cfpq_options_default(ctypes.byref(opt))
        opt.schedule, opt.path, opt.use_graph = schedule, path, int(bool(use_graph))
        opt.profile = int(bool(profile))
        opt.max_iter, opt.timeout_s = int(max_iter), float(timeout_s)
        opt.lengths = int(bool(lengths))
        opt.dense_tensor = int(bool(dense_tensor))
        opt.tensor_kind = int(tensor_kind)
        opt.row_begin, opt.row_end = int(row_begin), int(row_end)
        rec = _edges_struct(edges)
        h = ctypes.c_void_p()
        ptr = rec.ctypes.data_as(ctypes.POINTER(Edge)) if rec.size else None
        code = _lib().cfpq_create(grammar.cnf, self.n, ptr, rec.size, ctypes.byref(opt), ctypes.byref(h))
        _check(code, "cfpq_create")
        self._h = h
        self.status = None

    @property
    def handle(self):
        return self._h

    def solve(self, stream=None, check: bool = True) -> int:
        code = _lib().cfpq_solve(self._h, _stream_handle(stream))
        self.status = code
        if check:
            _check(code, "cfpq_solve")
        return code

    def _aid(self, A):
        return self.grammar.id(A) if isinstance(A, str) else int(A)

    def count(self, A) -> int:
        c = ctypes.c_size_t()
        _check(_lib().cfpq_count(self._h, self._aid(A), ctypes.byref(c)), "cfpq_count")
        return int(c.value)

    def triples(self, A) -> np.ndarray:
        """R_A as an (k, 3) uint32 array of (A, m, n) triples, sorted by (m, n)."""
        a = self._aid(A)
        c = ctypes.c_size_t()
        _check(_lib().cfpq_get(self._h, a, None, 0, ctypes.byref(c)), "cfpq_get")
        k = int(c.value)
        buf = _triple_rows(k)
        _check(_lib().cfpq_get(self._h, a, _triple_ptr(buf), k, ctypes.byref(c)), "cfpq_get")
        return buf[:k]

    def triples_all(self) -> np.ndarray:
        """Every relation as an (k, 3) uint32 array of (A, m, n), sorted (``cfpq_get_all``).
        The last solve's pair counters (seed pairs plus pairs the products added, each counted
        when its bit was first set) size the buffer, so one call usually does; a buffer that
        turns out too small takes the exact count from that call and a second one."""
        c = ctypes.c_size_t()
        st = Stats()
        _check(_lib().cfpq_stats_get(self._h, ctypes.byref(st)), "cfpq_stats_get")
        hint = max(0, int(st.seed_bits) + int(st.new_bits))
        if hint > 0:
            buf = _triple_rows(hint)
            rc = _lib().cfpq_get_all(self._h, _triple_ptr(buf), hint, ctypes.byref(c))
            if rc == OK:
                return buf[:int(c.value)]
            if rc != ERR_BUFFER:
                _check(rc, "cfpq_get_all")
        else:
            _check(_lib().cfpq_get_all(self._h, None, 0, ctypes.byref(c)), "cfpq_get_all")
        k = int(c.value)
        buf = _triple_rows(k)
        _check(_lib().cfpq_get_all(self._h, _triple_ptr(buf), k, ctypes.byref(c)), "cfpq_get_all")
        return buf[:k]

    def get(self, A) -> np.ndarray:
        """R_A as a sorted (k, 2) uint32 array of (m, n)."""
        a = self._aid(A)
        c = ctypes.c_size_t()
        _check(_lib().cfpq_get(self._h, a, None, 0, ctypes.byref(c)), "cfpq_get")
        k = int(c.value)
        buf = _triple_rows(k)
        _check(_lib().cfpq_get(self._h, a, _triple_ptr(buf), k, ctypes.byref(c)), "cfpq_get")
        return np.ascontiguousarray(buf[:k, 1:])

    def lengths(self, A):
        """Single-path semantics (``cfpq_get_lengths``): R_A as a sorted (k, 2) uint32 array of
        (m, n) and, per pair, the uint32 length of the walk it carries."""
        a = self._aid(A)
        c = ctypes.c_size_t()
        _check(_lib().cfpq_get_lengths(self._h, a, None, None, 0, ctypes.byref(c)), "cfpq_get_lengths")
        k = int(c.value)
        buf = _triple_rows(k)
        lens = np.empty(max(k, 1), dtype=np.uint32)
        _check(_lib().cfpq_get_lengths(self._h, a, _triple_ptr(buf),
                                       lens.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), k, ctypes.byref(c)),
               "cfpq_get_lengths")
        return np.ascontiguousarray(buf[:k, 1:]), lens[:k]

    def path(self, A, m: int, n: int):
        """Single-path semantics (``cfpq_get_path``): one walk from m to n whose labels A
        derives, as (nodes, labels): l + 1 uint32 node ids and l int32 terminal ids."""
        a = self._aid(A)
        c = ctypes.c_size_t()
        _check(_lib().cfpq_get_path(self._h, a, int(m), int(n), None, None, 0, ctypes.byref(c)), "cfpq_get_path")
        k = int(c.value)
        nodes = np.zeros(k + 1, dtype=np.uint32)
        labels = np.zeros(max(k, 1), dtype=np.int32)
        _check(_lib().cfpq_get_path(self._h, a, int(m), int(n), nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                    labels.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), k, ctypes.byref(c)),
               "cfpq_get_path")
        return nodes, labels[:k]

    def get_device(self, A, dev_ptr: int, cap: int) -> int:
        """Writes R_A as triples into device memory at dev_ptr (cap triples); returns |R_A|."""
        c = ctypes.c_size_t()
        _check(_lib().cfpq_get_device(self._h, self._aid(A), ctypes.c_void_p(dev_ptr), cap, ctypes.byref(c)),
               "cfpq_get_device")
        return int(c.value)

    def get_all_device(self, dev_ptr: int, cap: int) -> int:
        """Writes every relation as triples sorted by (A, m, n) into device memory at dev_ptr
        (cap triples; one host synchronisation); returns the number of triples."""
        c = ctypes.c_size_t()
        _check(_lib().cfpq_get_all_device(self._h, ctypes.c_void_p(dev_ptr) if dev_ptr else None, cap,
                                          ctypes.byref(c)), "cfpq_get_all_device")
        return int(c.value)

    # checkpoint and resume of the loop (cfpq_export_state / cfpq_import_state / cfpq_resume)
    def export_state(self) -> np.ndarray:
        """The loop's state (T, the next execution's delta, bitmaps, counts) as a uint8 array."""
        n = ctypes.c_size_t()
        _check(_lib().cfpq_state_size(self._h, ctypes.byref(n)), "cfpq_state_size")
        buf = np.empty(n.value, dtype=np.uint8)
        _check(_lib().cfpq_export_state(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.size), "cfpq_export_state")
        return buf

    def import_state(self, image: np.ndarray):
        image = np.ascontiguousarray(image, dtype=np.uint8)
        _check(_lib().cfpq_import_state(self._h, image.ctypes.data_as(ctypes.c_void_p), image.size),
               "cfpq_import_state")

    def resume(self, stream=None, more_executions: int = 0, check: bool = True) -> int:
        code = _lib().cfpq_resume(self._h, _stream_handle(stream), int(more_executions))
        self.status = code
        if check:
            _check(code, "cfpq_resume")
        return code

    # sharded solve by row blocks (contexts created with row_begin / row_end): the calls of
    # cfpq_block_*; the exchange between them is the caller's (see shard.py)
    @property
    def record_words(self) -> int:
        """32-bit words of one exchange record: non-terminal, row, then the row's n_pad / 32 words."""
        return 2 + ((self.n + 255) // 256 * 256) // 32

    def block_start(self, stream=None):
        _check(_lib().cfpq_block_start(self._h, _stream_handle(stream)), "cfpq_block_start")

    def block_products(self, stream=None):
        _check(_lib().cfpq_block_products(self._h, _stream_handle(stream)), "cfpq_block_products")

    def block_export(self, dev_ptr: int, cap_words: int, stream=None) -> int:
        """Packs this execution's new pairs of the context's rows into device memory; returns the
        words written (CfpqError ERR_BUFFER, with .words set, if cap_words is too small)."""
        w = ctypes.c_size_t()
        code = _lib().cfpq_block_export(self._h, ctypes.c_void_p(dev_ptr) if dev_ptr else None, cap_words,
                                        ctypes.byref(w), _stream_handle(stream))
        if code == ERR_BUFFER:
            err = CfpqError(code, "cfpq_block_export")
            err.words = int(w.value)
            raise err
        _check(code, "cfpq_block_export")
        return int(w.value)

    def block_import(self, dev_ptr: int, words: int, stream=None):
        _check(_lib().cfpq_block_import(self._h, ctypes.c_void_p(dev_ptr) if dev_ptr else None, words,
                                        _stream_handle(stream)), "cfpq_block_import")

    def block_finish(self, stream=None) -> bool:
        """Ends the execution; True if the loop goes on."""
        ch = ctypes.c_int32()
        _check(_lib().cfpq_block_finish(self._h, _stream_handle(stream), ctypes.byref(ch)), "cfpq_block_finish")
        return bool(ch.value)

    def stats(self) -> dict:
        s = Stats()
        _check(_lib().cfpq_stats_get(self._h, ctypes.byref(s)), "cfpq_stats_get")
        return s.as_dict()

    def close(self):
        h = getattr(self, "_h", None)
        if h and _LIB is not None:
            _LIB.cfpq_destroy(h)
        self._h = None

    def __del__(self):
        self.close()


def extract_pairs_noalloc(bits_ptr: int, n_rows: int, n_cols: int, row_words: int, A: int, out_ptr: int,
                          cap: int, stream=None) -> int:
    """Pairs of a caller-owned bit-packed device matrix written as (A, m, n) triples into a
    caller-owned device buffer, without any allocation by the library
    (``cfpq_extract_pairs_noalloc``); returns the number of pairs."""
    c = ctypes.c_size_t()
    code = _lib().cfpq_extract_pairs_noalloc(ctypes.c_void_p(bits_ptr), n_rows, n_cols, row_words, A,
                                             ctypes.c_void_p(out_ptr) if out_ptr else None, cap, ctypes.byref(c),
                                             _stream_handle(stream))
    _check(code, "cfpq_extract_pairs_noalloc")
    return int(c.value)


class Server:
    """Continuous-batching server (``cfpq_server_*``): submit queries at any time, call
    ``step()`` to admit, advance and retire; results of finished queries stay on the host."""

    def __init__(self, hbm_budget_bytes: int = 0, rounds_per_step: int = 8, max_resident: int = 0):
        o = ServerOptions()
        _lib().cfpq_server_options_default(ctypes.byref(o))
        o.hbm_budget_bytes, o.rounds_per_step, o.max_resident = int(hbm_budget_bytes), int(rounds_per_step), \
            int(max_resident)
        h = ctypes.c_void_p()
        _check(_lib().cfpq_server_create(ctypes.byref(o), ctypes.byref(h)), "cfpq_server_create")
        self._h = h

    def submit(self, grammar: Grammar, n: int, edges, schedule: int = SCHED_INPLACE) -> int:
        rec = _edges_struct(edges)
        t = ctypes.c_int64()
        ptr = rec.ctypes.data_as(ctypes.POINTER(Edge)) if rec.size else None
        _check(_lib().cfpq_server_submit(self._h, grammar.cnf, int(n), ptr, rec.size, schedule, ctypes.byref(t)),
               "cfpq_server_submit")
        return int(t.value)

    def step(self) -> int:
        c = ctypes.c_int32()
        _check(_lib().cfpq_server_step(self._h, ctypes.byref(c)), "cfpq_server_step")
        return int(c.value)

    def completed(self) -> list:
        c = ctypes.c_size_t()
        _check(_lib().cfpq_server_completed(self._h, None, 0, ctypes.byref(c)), "cfpq_server_completed")
        buf = (ctypes.c_int64 * max(1, c.value))()
        _check(_lib().cfpq_server_completed(self._h, buf, c.value, ctypes.byref(c)), "cfpq_server_completed")
        return [int(buf[i]) for i in range(c.value)]

    def info(self, ticket: int) -> dict:
        q = QueryInfo()
        _check(_lib().cfpq_server_query_info(self._h, ticket, ctypes.byref(q)), "cfpq_server_query_info")
        return {"state": q.state, "status": q.status, "iterations": q.iterations, "n_nonterm": q.n_nonterm}

    def result(self, ticket: int, A: int) -> np.ndarray:
        """R_A of a finished query as a sorted (k, 2) uint32 array of (m, n)."""
        c = ctypes.c_size_t()
        _check(_lib().cfpq_server_result(self._h, ticket, A, None, 0, ctypes.byref(c)), "cfpq_server_result")
        k = int(c.value)
        buf = _triple_rows(k)
        _check(_lib().cfpq_server_result(self._h, ticket, A, _triple_ptr(buf), k, ctypes.byref(c)),
               "cfpq_server_result")
        return np.ascontiguousarray(buf[:k, 1:])

    def release(self, ticket: int):
        _check(_lib().cfpq_server_release(self._h, ticket), "cfpq_server_release")

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib().cfpq_server_stats_get(self._h, ctypes.byref(st)), "cfpq_server_stats_get")
        return st.as_dict()

    def close(self):
        h = getattr(self, "_h", None)
        if h and _LIB is not None:
            _LIB.cfpq_server_destroy(h)
        self._h = None

    def __del__(self):
        self.close()


def _handles(queries):
    return (ctypes.c_void_p * len(queries))(*[q.handle.value for q in queries])


def solve_batch(queries, stream=None, check: bool = True, tuning: BatchTuning | None = None) -> int:
    """Solves many queries in one grouped persistent launch (``cfpq_solve_batch``, or
    ``cfpq_solve_batch_tuned`` under an explicit configuration)."""
    arr = _handles(queries)
    if tuning is None:
        code = _lib().cfpq_solve_batch(arr, len(queries), _stream_handle(stream))
    else:
        code = _lib().cfpq_solve_batch_tuned(arr, len(queries), ctypes.byref(tuning), _stream_handle(stream))
    for q in queries:
        q.status = code
    if check:
        _check(code, "cfpq_solve_batch")
    return code


def batch_tuning_default() -> BatchTuning:
    t = BatchTuning()
    _lib().cfpq_batch_tuning_default(ctypes.byref(t))
    return t


def batch_tuning() -> BatchTuning:
    """The configuration batched solves and serving steps use now."""
    t = BatchTuning()
    _check(_lib().cfpq_batch_tuning_get(ctypes.byref(t)), "cfpq_batch_tuning_get")
    return t


def set_batch_tuning(t: BatchTuning) -> None:
    _check(_lib().cfpq_batch_tuning_set(ctypes.byref(t)), "cfpq_batch_tuning_set")


def autotune_batch(queries, stream=None):
    """Times candidate launch configurations on this batch (``cfpq_autotune_batch``),
    installs the best and returns (BatchTuning, report dict)."""
    best, rep = BatchTuning(), TuneReport()
    code = _lib().cfpq_autotune_batch(_handles(queries), len(queries), _stream_handle(stream), ctypes.byref(best),
                                      ctypes.byref(rep))
    for q in queries:
        q.status = code
    _check(code, "cfpq_autotune_batch")
    return best, {"trials": rep.trials, "default_ms": rep.default_ms, "best_ms": rep.best_ms}


BATCH_PHASES = ("start", "scan", "products", "jacobi_merge", "tails", "tables")
BATCH_PROFILE_ROUNDS = 64


def batch_last_profile() -> dict:
    """Per-phase device time (ms) and round count of the last batched launch."""
    arr = (ctypes.c_double * len(BATCH_PHASES))()
    per_round = (ctypes.c_double * BATCH_PROFILE_ROUNDS)()
    rounds = ctypes.c_int64()
    _check(_lib().cfpq_batch_last_profile(arr, len(BATCH_PHASES), ctypes.byref(rounds), per_round,
                                          BATCH_PROFILE_ROUNDS), "cfpq_batch_last_profile")
    out = {name: arr[i] for i, name in enumerate(BATCH_PHASES)}
    out["rounds"] = int(rounds.value)
    out["round_products"] = [per_round[i] for i in range(min(out["rounds"], BATCH_PROFILE_ROUNDS))]
    return out


def measure_mma_sync_peaks() -> dict:
    """Measured mma.sync s8 and b1 (AND/popc) tensor throughput of the current device, TOPS."""
    s8, b1 = ctypes.c_double(), ctypes.c_double()
    _check(_lib().cfpq_measure_mma_sync_peaks(ctypes.byref(s8), ctypes.byref(b1)), "cfpq_measure_mma_sync_peaks")
    return {"s8_tops": s8.value, "b1_tops": b1.value}


def measure_tensor_peaks() -> dict:
    """Measured dense rate of the tcgen05 kinds f8f6f4 (E4M3) and mxf4 (E2M1, unit scales) in
    the product kernels' tile shape, TFLOP/s and ops per SM clock, with the exactness check."""
    p = TensorPeaks()
    _check(_lib().cfpq_measure_tensor_peaks(ctypes.byref(p)), "cfpq_measure_tensor_peaks")
    return p.as_dict()


def trim_memory(keep_bytes: int = 0):
    """Hands the device memory that destroyed queries left in the library's pool on the
    current device back to the system, keeping at most keep_bytes (``cfpq_trim_memory``)."""
    _check(_lib().cfpq_trim_memory(int(keep_bytes)), "cfpq_trim_memory")
