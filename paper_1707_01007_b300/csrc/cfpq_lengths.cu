// Single-path semantics (Section 5): next to the Boolean closure, every pair (A, i, j) carries
// the length l_A(i, j) of one walk from i to j whose labels A derives.
//
//   seed        an edge (i, x, j) gives every A -> x the length 1; A -> eps gives (m, m) the
//               length 0 (the empty walk)
//   execution   a pair (A, i, j) that a loop execution adds through A -> B C and a middle node
//               k gets l_B(i, k) + l_C(k, j), read from the matrices before the execution; the
//               length of a pair is set once, by the execution that adds the pair, and kept
//
// The paper leaves open which length is kept when one execution derives the same new pair
// through several productions or middle nodes; this engine keeps the smallest, so the result
// is unique and does not depend on the order in which the device finds the derivations.
//
// Layout: one uint32 plane per non-terminal next to T, L[A][i * n_pad + j]. The search for the
// middle nodes k of a pair (i, j) intersects row i of T_B with column j of T_C; for that the
// seed and the Jacobi merge (k_merge) keep T^T up to date pair by pair, with a word summary of
// T and of T^T (one bit per 32-bit word, SW words per row), so that only words that are
// non-zero on both sides are read. A length cell is only
// written when its pair enters T_A and only read while the pair is in T_A, so the planes are
// never cleared. The loop runs under the Jacobi schedule (T_{k+1} = T_k u T_k x T_k): after
// every product of an execution has written its new pairs to the delta plane N and before
// N is merged into T, k_lengths reads N (the new pairs) and the unchanged T of the previous
// execution, which is exactly the matrices the lengths must come from.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "cfpq_device.cuh"
#include "cfpq_internal.h"
#include "cfpq_lengths.cuh"

namespace cfpq {

// Matrix initialisation of the lengths; runs after k_seed (which sets the same pairs in T).
// eps_mask bit a: A -> eps, so a loop edge (m, x, m) of a nullable A is left to the empty walk
// (length 0). Several edges of one pair store their labels in any order here; the next
// kernel keeps the smallest.
__global__ void k_seed_lengths(const QDesc *qd, uint32_t *L, uint32_t *Wit, uint64_t lplane,
                               unsigned long long eps_mask) {
    const QDesc &q = *qd;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = tid; e < q.n_edges; e += nth) {
        const cfpq_edge ed = q.edges[e];
        for (int u = 0; u < q.n_unary; u++)
            if (q.unary[u].y == ed.label) {
                const int a = q.unary[u].x;
                if (ed.src == ed.dst && ((eps_mask >> a) & 1ull)) continue;
                const uint64_t cell = (uint64_t)a * lplane + (uint64_t)ed.src * q.n_pad + ed.dst;
                L[cell] = 1u;
                Wit[cell] = kWitEdge | (uint32_t)ed.label;
            }
    }
    for (uint64_t t = tid; t < (uint64_t)q.n_eps * q.n; t += nth) {
        const int a = q.eps[t / q.n];
        const uint64_t cell = (uint64_t)a * lplane + (t % q.n) * q.n_pad + t % q.n;
        L[cell] = 0u;
        Wit[cell] = kWitEps;
    }
}

// Second pass over the edges: the smallest label among several edges of one pair.
__global__ void k_seed_witness_min(const QDesc *qd, uint32_t *Wit, uint64_t lplane, unsigned long long eps_mask) {
    const QDesc &q = *qd;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < q.n_edges;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const cfpq_edge ed = q.edges[e];
        for (int u = 0; u < q.n_unary; u++)
            if (q.unary[u].y == ed.label) {
                const int a = q.unary[u].x;
                if (ed.src == ed.dst && ((eps_mask >> a) & 1ull)) continue;
                atomicMin(&Wit[(uint64_t)a * lplane + (uint64_t)ed.src * q.n_pad + ed.dst], kWitEdge | (uint32_t)ed.label);
            }
    }
}

// Persistent grid over the pairs the execution added (lengths_of_new_pairs).
__global__ void __launch_bounds__(256, 3) k_lengths(const QDesc *qd, uint32_t *L, uint32_t *Wit, uint64_t lplane) {
    lengths_of_new_pairs(*qd, L, Wit, lplane);
}

// Rebuilds the walk of (a, m, n) from the recorded derivation steps, depth first, left child
// first (one thread). Stack entries (A, i, j, offset of the sub-walk's first edge). Every
// child was derived in an earlier loop execution than its parent, so the stack never holds
// more entries than executions + 1; stack_cap and max_steps only guard against a corrupt
// state. status: 0 ok, 1 stack full, 2 step limit, 3 inconsistent witness.
__global__ void k_path(const QDesc *qd, const uint32_t *L, const uint32_t *Wit, uint64_t lplane, int a, uint32_t m,
                       uint32_t n, uint32_t len, uint32_t *nodes, int32_t *labels, uint4 *stack, uint32_t stack_cap,
                       unsigned long long max_steps, uint32_t *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const QDesc &q = *qd;
    const uint64_t np = q.n_pad;
    nodes[0] = m;
    uint32_t sp = 0;
    stack[sp++] = make_uint4((uint32_t)a, m, n, 0u);
    unsigned long long steps = 0;
    while (sp > 0) {
        if (++steps > max_steps) { *status = 2u; return; }
        const uint4 e = stack[--sp];
        const uint32_t w = Wit[(uint64_t)e.x * lplane + (uint64_t)e.y * np + e.z];
        if (w == kWitEps) continue;
        if (w & kWitEdge) {
            if (e.w >= len) { *status = 3u; return; }
            labels[e.w] = (int32_t)(w & ~kWitEdge);
            nodes[e.w + 1] = e.z;
            continue;
        }
        const uint32_t r = w >> kWitK, k = w & ((1u << kWitK) - 1u);
        if (r >= (uint32_t)q.n_rules || k >= q.n) { *status = 3u; return; }
        const int B = q.rules[r].b, C = q.rules[r].c;
        const uint32_t lb = L[(uint64_t)B * lplane + (uint64_t)e.y * np + k];
        if ((unsigned long long)e.w + lb > len) { *status = 3u; return; }
        if (sp + 2 > stack_cap) { *status = 1u; return; }
        stack[sp++] = make_uint4((uint32_t)C, k, e.z, e.w + lb);
        stack[sp++] = make_uint4((uint32_t)B, e.y, k, e.w);
    }
    *status = 0u;
}

// Lengths of extracted triples: out[t] = L[A][m * n_pad + n].
__global__ void k_triple_lengths(const cfpq_triple *tr, uint64_t count, const uint32_t *L, uint64_t lplane,
                                 uint32_t n_pad, uint32_t *out) {
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (uint64_t)gridDim.x * blockDim.x) {
        const cfpq_triple x = tr[t];
        out[t] = __ldg(L + (uint64_t)x.A * lplane + (uint64_t)x.m * n_pad + x.n);
    }
}

static unsigned long long eps_mask(const cfpq_ctx *c) {
    unsigned long long m = 0;
    for (int32_t a : c->h_eps) m |= 1ull << a;
    return m;
}

int lengths_enqueue_seed(cfpq_ctx *c, cudaStream_t s) {
    const uint64_t work = std::max<uint64_t>(c->n_edges, (uint64_t)c->n_eps_rules * c->n);
    const uint32_t blocks = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(1, (work + 255) / 256), 148ull * 16);
    k_seed_lengths<<<blocks, 256, 0, s>>>(c->d_q, c->d_L, c->d_Wit, c->lplane, eps_mask(c));
    k_seed_witness_min<<<blocks, 256, 0, s>>>(c->d_q, c->d_Wit, c->lplane, eps_mask(c));
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

// Persistent grid of the length kernels: the SMs times the resident blocks of k_lengths (the
// kernel of the two with the most registers).
static int ensure_len_grid(cfpq_ctx *c) {
    if (c->len_grid) return CFPQ_OK;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CFPQ_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lengths, 256, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    c->len_grid = std::max(1, sms) * per_sm;
    return CFPQ_OK;
}

int lengths_enqueue_iteration(cfpq_ctx *c, cudaStream_t s) {
    const int rc = ensure_len_grid(c);
    if (rc != CFPQ_OK) return rc;
    const uint64_t blocks_needed = ((uint64_t)c->n_nt * c->n + kLenWarps - 1) / kLenWarps;
    const uint32_t blocks = (uint32_t)std::min<uint64_t>((uint64_t)c->len_grid, std::max<uint64_t>(1, blocks_needed));
    k_lengths<<<blocks, 256, 0, s>>>(c->d_q, c->d_L, c->d_Wit, c->lplane);
    c->iter_launches++;
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

int lengths_of_triples(cfpq_ctx *c, const cfpq_triple *d_tr, size_t count, uint32_t *d_out, cudaStream_t s) {
    if (count == 0) return CFPQ_OK;
    const uint32_t blocks = (uint32_t)std::min<uint64_t>((count + 255) / 256, 148ull * 32);
    k_triple_lengths<<<blocks, 256, 0, s>>>(d_tr, count, c->d_L, c->lplane, c->n_pad, d_out);
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

int lengths_rules_ok(const cfpq_ctx *c) { return c->rules.size() < kMaxLenRules; }

// One walk of (A, m, n) into host memory (cfpq_get_path after its checks).
int lengths_path(cfpq_ctx *c, int32_t A, uint32_t m, uint32_t n, uint32_t len, uint32_t *nodes, int32_t *labels) {
    cudaStream_t s = c->last_stream;
    const uint32_t stack_cap = (uint32_t)std::min<uint64_t>((uint64_t)c->stats.iterations + 8, 1ull << 30);
    const unsigned long long max_steps = (2ull * len + 1ull) * ((unsigned long long)c->stats.iterations + 1ull) + 16ull;
    const size_t b_nodes = ((size_t)len + 1) * sizeof(uint32_t), b_labels = std::max<size_t>(1, len) * sizeof(int32_t);
    const size_t b_stack = (size_t)stack_cap * sizeof(uint4);
    const size_t off_labels = (b_nodes + 255) / 256 * 256, off_stack = off_labels + (b_labels + 255) / 256 * 256;
    const size_t off_status = off_stack + (b_stack + 255) / 256 * 256;
    char *buf = nullptr;
    if (cudaMalloc(&buf, off_status + 256) != cudaSuccess) {
        cudaGetLastError();
        return CFPQ_ERR_NOMEM;
    }
    uint32_t *d_nodes = reinterpret_cast<uint32_t *>(buf);
    int32_t *d_labels = reinterpret_cast<int32_t *>(buf + off_labels);
    uint4 *d_stack = reinterpret_cast<uint4 *>(buf + off_stack);
    uint32_t *d_status = reinterpret_cast<uint32_t *>(buf + off_status);
    uint32_t status = 4u;
    int rc = CFPQ_OK;
    k_path<<<1, 32, 0, s>>>(c->d_q, c->d_L, c->d_Wit, c->lplane, A, m, n, len, d_nodes, d_labels, d_stack, stack_cap,
                            max_steps, d_status);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&status, d_status, sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(nodes, d_nodes, b_nodes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        (len && cudaMemcpyAsync(labels, d_labels, (size_t)len * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess)
        rc = CFPQ_ERR_CUDA;
    cudaFree(buf);
    if (rc == CFPQ_OK && status != 0u) rc = CFPQ_ERR_CUDA;
    return rc;
}

}  // namespace cfpq
