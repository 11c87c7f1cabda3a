"""Allocation-free extraction (cfpq_extract_pairs_noalloc) against the allocating path.

Callers that cannot allocate device memory (an external allocator owns the device heap,
or cudaMalloc is not allowed on their path) pass a bit-packed relation matrix and an
output buffer that they own; the library then uses only its fixed device scratch array.
Its output must equal what the allocating entry point (cfpq_get_device) returns for the
same relation, on consecutive calls: the shared scratch array keeps the previous call's
contents, so a second call must not be affected by the first."""
import ctypes

import numpy as np
import pytest

import cfpq_synth as synth
import paper_1707_01007_b300 as eng

pytestmark = pytest.mark.gpu

MAX_ROWS = 65536  # CFPQ_NOALLOC_MAX_ROWS


def bit_matrix(pairs, n_rows, row_words):
    m = np.zeros((n_rows, row_words), dtype=np.uint32)
    if len(pairs):
        r = pairs[:, 0].astype(np.int64)
        c = pairs[:, 1].astype(np.int64)
        np.bitwise_or.at(m, (r, c // 32), np.left_shift(np.uint32(1), (c % 32).astype(np.uint32)))
    return m


def reference_triples(q, name):
    """R_name through the allocating device entry point, copied back to the host."""
    import torch

    k = q.count(name)
    buf = torch.empty(max(1, k) * 3, dtype=torch.int32, device="cuda")
    assert q.get_device(name, buf.data_ptr(), max(1, k)) == k
    torch.cuda.synchronize()
    return buf[: 3 * k].view(-1, 3).cpu().numpy()


def run_noalloc(bits_np, n_rows, n_cols, a, cap):
    import torch

    bits = torch.from_numpy(bits_np.view(np.int32)).cuda()
    out = torch.full((max(1, cap) * 3,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    got = eng.extract_pairs_noalloc(bits.data_ptr(), n_rows, n_cols, bits_np.shape[1], a, out.data_ptr(),
                                    max(1, cap), stream)
    torch.cuda.synchronize()
    return got, out[: 3 * got].view(-1, 3).cpu().numpy()


def test_noalloc_equals_allocating_extraction_twice():
    graph = synth.hierarchy(1500, 450, seed=5)
    g = eng.Grammar(synth.GRAMMAR_Q1, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, timeout_s=120.0)
    q.solve()
    row_words = (graph.n + 31) // 32 + 1  # one spare word per row: columns >= n must be ignored
    for name in ["S", "X", "<ty_r>", "Y"]:
        ref = reference_triples(q, name)
        bits = bit_matrix(ref[:, 1:], graph.n, row_words)
        bits[:, -1] |= np.uint32(0xFFFFFFFF)  # bits beyond n_cols: not part of the relation
        for _ in range(2):  # two calls in a row share the scratch array
            got, out = run_noalloc(bits, graph.n, graph.n, g.id(name), len(ref))
            assert got == len(ref)
            assert np.array_equal(out, ref)


def test_noalloc_large_then_small():
    rng = np.random.default_rng(1)
    big = (rng.random((4000, 126)) < 0.02).astype(np.uint8)
    small = (rng.random((37, 2)) < 0.3).astype(np.uint8)
    for mat in (big, small, big):
        n_rows, n_cols = mat.shape
        pairs = np.argwhere(mat)
        bits = bit_matrix(pairs, n_rows, (n_cols + 31) // 32)
        got, out = run_noalloc(bits, n_rows, n_cols, 3, len(pairs))
        assert got == len(pairs)
        exp = np.concatenate([np.full((len(pairs), 1), 3), pairs], axis=1).astype(np.int32)
        assert np.array_equal(out, exp)


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch

    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    c = ctypes.c_size_t(123)
    code = eng.library().cfpq_extract_pairs_noalloc(ctypes.c_void_p(dummy.data_ptr()), MAX_ROWS + 1, 32, 1, 0,
                                                    None, 0, ctypes.byref(c), None)
    assert code == eng.ERR_INVALID
    code = eng.library().cfpq_extract_pairs_noalloc(ctypes.c_void_p(dummy.data_ptr()), 1, 64, 1, 0, None, 0,
                                                    ctypes.byref(c), None)
    assert code == eng.ERR_INVALID  # n_cols wider than the rows


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises its stream and reads the count on the host, which a stream
    capture cannot contain: on a capturing stream it is refused before any device work, the
    capture can still be ended, and the next ordinary call works."""
    import torch

    graph = synth.hierarchy(600, 180, seed=2)
    g = eng.Grammar(synth.GRAMMAR_QSC, graph.labels)
    q = eng.Query(g, graph.n, graph.edges, timeout_s=120.0)
    q.solve()
    ref = reference_triples(q, "S")
    row_words = (graph.n + 31) // 32
    bits_np = bit_matrix(ref[:, 1:], graph.n, row_words)
    bits = torch.from_numpy(bits_np.view(np.int32)).cuda()
    out = torch.zeros(max(1, len(ref)) * 3, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    c = ctypes.c_size_t(0)
    lib = eng.library()
    cg = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(cg, stream=side):
        out.add_(0)  # one captured operation, so that the graph is not empty
        code = lib.cfpq_extract_pairs_noalloc(ctypes.c_void_p(bits.data_ptr()), graph.n, graph.n, row_words,
                                              g.id("S"), ctypes.c_void_p(out.data_ptr()), len(ref),
                                              ctypes.byref(c), ctypes.c_void_p(side.cuda_stream))
    assert code == eng.ERR_INVALID
    torch.cuda.synchronize()
    got, arr = run_noalloc(bits_np, graph.n, graph.n, g.id("S"), len(ref))
    assert got == len(ref) and np.array_equal(arr, ref)
