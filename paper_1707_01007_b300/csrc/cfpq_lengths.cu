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

namespace cfpq {

// Derivation step of a pair (one uint32 per cell beside its length, the "witness"), from
// which cfpq_get_path rebuilds the walk: the empty walk (A -> eps), an edge with its label,
// or production rules[r] with middle node k. Ordered so that a smaller word is preferred.
constexpr uint32_t kWitEps = 0x40000000u;             // (m, m) by A -> eps: length 0
constexpr uint32_t kWitEdge = 0x80000000u;            // | label: an edge (m, label, n), length 1
constexpr uint32_t kWitK = 17;                        // split: (r << 17) | k, r < 8192
constexpr uint32_t kMaxLenRules = 1u << (30 - kWitK);

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

// Summary words of a row taken per step of the middle-node search: kSumVec 16-byte loads.
constexpr int kSumVec = 2;

// Length of one new pair (A, i, j) from the productions r0 .. r1 - 1 of A (one lane, one
// pair). The middle nodes k under A -> B C are the set bits of row i of T_B AND row j of TT_C
// (column j of T_C): the two rows' word summaries are ANDed 4 kSumVec words at a time
// (vector loads), and only the words both flag are read and ANDed. Returns the minimum of
// l_B(i, k) + l_C(k, j) (UINT64_MAX if there is no middle node) and, in *wit, the production
// index and middle node of the first minimum found (smallest index, then smallest k).
__device__ __forceinline__ unsigned long long pair_length(const QDesc &q, const uint32_t *__restrict__ L,
                                                          uint64_t lplane, int r0, int r1, uint32_t i, uint32_t j,
                                                          unsigned *hits, uint32_t *wit) {
    const uint32_t W = q.W, np = q.n_pad, SW = q.SW;
    unsigned long long best = ~0ull;
    *wit = 0u;
    for (int r = r0; r < r1; r++) {
        const int B = q.rules[r].b, C = q.rules[r].c;
        const uint4 *sumB = reinterpret_cast<const uint4 *>(q.Tsum + ((uint64_t)B * np + i) * SW);
        const uint4 *sumC = reinterpret_cast<const uint4 *>(q.TTsum + ((uint64_t)C * np + j) * SW);
        const uint32_t *rowB = q.T + (uint64_t)B * q.plane + (uint64_t)i * W;
        const uint32_t *colC = q.TT + (uint64_t)C * q.plane + (uint64_t)j * W;
        const uint32_t *LB = L + (uint64_t)B * lplane + (uint64_t)i * np;
        const uint32_t *LC = L + (uint64_t)C * lplane + j;
        for (uint32_t s0 = 0; s0 < SW; s0 += 4u * kSumVec) {
            uint4 b[kSumVec], c[kSumVec];
#pragma unroll
            for (int t = 0; t < kSumVec; t++) {
                const bool in = s0 + 4u * t < SW;
                b[t] = in ? __ldcg(sumB + s0 / 4 + t) : make_uint4(0u, 0u, 0u, 0u);
                c[t] = in ? __ldcg(sumC + s0 / 4 + t) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int t = 0; t < kSumVec; t++) {
                const uint32_t xs[4] = {b[t].x & c[t].x, b[t].y & c[t].y, b[t].z & c[t].z, b[t].w & c[t].w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    uint32_t x = xs[e];  // words flagged in row i of T_B and in column j of T_C
                    while (x) {
                        const uint32_t wk = (s0 + 4u * t + (uint32_t)e) * 32u + (uint32_t)(__ffs(x) - 1);
                        x &= x - 1;
                        uint32_t kw = __ldcg(rowB + wk) & __ldcg(colC + wk);
                        while (kw) {
                            const uint32_t k = wk * 32u + (uint32_t)(__ffs(kw) - 1);
                            kw &= kw - 1;
                            const unsigned long long cand =
                                (unsigned long long)__ldcg(LB + k) + __ldcg(LC + (uint64_t)k * np);
                            if (cand < best) {  // productions, then k, ascending: the first minimum is kept
                                best = cand;
                                *wit = ((uint32_t)r << kWitK) | k;
                            }
                            (*hits)++;
                        }
                    }
                }
            }
        }
    }
    return best;
}

// Pairs queued per warp before the lanes take one each (two rounds of 32 fit).
constexpr int kLenQ = 64;
constexpr int kLenWarps = 8;
constexpr int kScanU = 4;  // 32-word chunks of a row of N loaded together

// Persistent grid. Warp g scans the rows (A, i) = g, g + warps, ... of the n_nt x n row space
// whose bit in the new delta's row bitmap is set (its lanes test 32 of those rows at once); the
// bits of N_A's row i are exactly the pairs this execution adds (read before the merge). Each new pair goes into the warp's queue in
// shared memory (every lane still holding bits gives one per round); whenever 32 are queued,
// every lane computes one pair's length, so the lanes stay busy however the new pairs are
// spread over rows and words.
__global__ void __launch_bounds__(256, 3) k_lengths(const QDesc *qd, uint32_t *L, uint32_t *Wit, uint64_t lplane) {
    __shared__ uint32_t q_i[kLenWarps][kLenQ], q_j[kLenWarps][kLenQ];
    __shared__ uint8_t q_a[kLenWarps][kLenQ];
    __shared__ int2 grp[kMaxNT];  // productions of each left-hand side: [x, y)
    const QDesc &q = *qd;
    if (threadIdx.x < (unsigned)q.n_nt) grp[threadIdx.x] = q.nt_rules[threadIdx.x];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t gwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t parity = (uint32_t)(q.st->iter & 1ull);
    const uint32_t *NR = parity ? q.R0 : q.R1;
    const uint32_t *Nall = parity ? q.X0 : q.X1;
    const uint32_t W = q.W;
    const unsigned lt = (1u << lane) - 1u;
    unsigned hits = 0;
    int fill = 0;  // warp-uniform queue length

    // every lane takes queue entry `lane` (if it exists) and writes its pair's length
    auto run = [&](int cnt) {
        __syncwarp();
        if (lane < cnt) {
            const int a = q_a[warp][lane];
            const uint32_t i = q_i[warp][lane], j = q_j[warp][lane];
            uint32_t wit;
            const unsigned long long best = pair_length(q, L, lplane, grp[a].x, grp[a].y, i, j, &hits, &wit);
            const uint64_t cell = (uint64_t)a * lplane + (uint64_t)i * q.n_pad + j;
            L[cell] = best >= 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)best;
            Wit[cell] = wit;
        }
        __syncwarp();
    };

    // rows of this warp: g = gwarp + m * gwarps; lane l tests row m = 32 t + l of round t
    const uint64_t total = (uint64_t)q.n_nt * q.n;
    for (uint64_t base = gwarp; base < total; base += 32ull * gwarps) {
        const uint64_t mine = base + (uint64_t)lane * gwarps;
        bool flagged = false;
        if (mine < total) {
            const int a = (int)(mine / q.n);
            flagged = grp[a].x >= 0 && test_bit(NR + (uint64_t)a * W, (uint32_t)(mine % q.n));
        }
        unsigned rowmask = __ballot_sync(0xffffffffu, flagged);
        while (rowmask) {
            const int src = __ffs(rowmask) - 1;
            rowmask &= rowmask - 1;
            const uint64_t g = base + (uint64_t)src * gwarps;
            const int a = (int)(g / q.n);
            const uint32_t i = (uint32_t)(g % q.n);
            const uint32_t *N = Nall + (uint64_t)a * q.plane + (uint64_t)i * W;
            for (uint32_t w0 = 0; w0 < W; w0 += 32u * kScanU) {
                uint32_t nw[kScanU];
#pragma unroll
                for (int u = 0; u < kScanU; u++) {
                    const uint32_t w = w0 + 32u * u + lane;
                    nw[u] = w < W ? __ldcg(N + w) : 0u;
                }
#pragma unroll
                for (int u = 0; u < kScanU; u++) {
                    uint32_t x = nw[u];
                    const uint32_t jb = (w0 + 32u * u + lane) * 32u;
                    for (;;) {
                        const unsigned m = __ballot_sync(0xffffffffu, x != 0u);
                        if (!m) break;
                        if (x) {
                            const int pos = fill + __popc(m & lt);
                            q_a[warp][pos] = (uint8_t)a;
                            q_i[warp][pos] = i;
                            q_j[warp][pos] = jb + (uint32_t)(__ffs(x) - 1);
                            x &= x - 1;
                        }
                        fill += __popc(m);
                        if (fill >= 32) {
                            run(32);
                            if (lane < fill - 32) {  // move the rest (at most 31) to the front
                                q_a[warp][lane] = q_a[warp][32 + lane];
                                q_i[warp][lane] = q_i[warp][32 + lane];
                                q_j[warp][lane] = q_j[warp][32 + lane];
                            }
                            __syncwarp();
                            fill -= 32;
                        }
                    }
                }
            }
        }
    }
    if (fill > 0) run(fill);
    if (q.profile) {
        unsigned long long sp = hits;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o);
        if (lane == 0 && sp) atomicAdd(&q.st->len_splits, sp);
    }
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
