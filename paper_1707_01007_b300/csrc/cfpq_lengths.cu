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
// Layout: one uint32 plane per non-terminal next to T, L[A][i * n_pad + j]. A cell is only
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

// Matrix initialisation of the lengths; runs after k_seed (which sets the same pairs in T).
// eps_mask bit a: A -> eps, so a loop edge (m, x, m) of a nullable A keeps the length 0.
__global__ void k_seed_lengths(const QDesc *qd, uint32_t *L, uint64_t lplane, unsigned long long eps_mask) {
    const QDesc &q = *qd;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = tid; e < q.n_edges; e += nth) {
        const cfpq_edge ed = q.edges[e];
        for (int u = 0; u < q.n_unary; u++)
            if (q.unary[u].y == ed.label) {
                const int a = q.unary[u].x;
                const uint32_t len = (ed.src == ed.dst && ((eps_mask >> a) & 1ull)) ? 0u : 1u;
                L[(uint64_t)a * lplane + (uint64_t)ed.src * q.n_pad + ed.dst] = len;
            }
    }
    for (uint64_t t = tid; t < (uint64_t)q.n_eps * q.n; t += nth) {
        const int a = q.eps[t / q.n];
        const uint64_t m = t % q.n;
        L[(uint64_t)a * lplane + m * q.n_pad + m] = 0u;
    }
}

// Middle nodes taken per step of the split loop: their T_C words are loaded together, then
// their lengths, so that a warp keeps several independent loads in flight.
constexpr int kSplitU = 4;

// Lengths of the new pairs (A, i, 32 w + lane) flagged in `bits` (one bit per lane), for the
// productions r0 .. r1 - 1 of A. The warp walks the set bits k of row i of T_B (warp-uniform);
// for each k one word of T_C (row k, word w) says which lanes' j have (k, j) in T_C; those
// lanes take l_B(i, k) + l_C(k, j). Returns the lane's minimum (UINT64_MAX if it has no pair).
__device__ __forceinline__ unsigned long long min_split(const QDesc &q, const uint32_t *__restrict__ L, uint64_t lplane,
                                                        int r0, int r1, uint32_t i, uint32_t w, uint32_t bits,
                                                        int lane, unsigned long long *splits) {
    const uint32_t W = q.W, np = q.n_pad;
    const uint32_t j = w * 32u + (uint32_t)lane;
    const bool mine = (bits >> lane) & 1u;
    unsigned long long best = ~0ull;
    unsigned hits = 0;
    for (int r = r0; r < r1; r++) {
        const int B = q.rules[r].b, C = q.rules[r].c;
        const uint32_t *rowB = q.T + (uint64_t)B * q.plane + (uint64_t)i * W;
        const uint32_t *TC = q.T + (uint64_t)C * q.plane + w;
        const uint32_t *LB = L + (uint64_t)B * lplane + (uint64_t)i * np;
        const uint32_t *LC = L + (uint64_t)C * lplane + j;
        for (uint32_t w0 = 0; w0 < W; w0 += 32) {
            const uint32_t bw = (w0 + lane < W) ? __ldcg(rowB + w0 + lane) : 0u;
            unsigned nz = __ballot_sync(0xffffffffu, bw != 0u);
            uint32_t x = 0, kb = 0;
            while (nz || x) {
                uint32_t k[kSplitU];
#pragma unroll
                for (int u = 0; u < kSplitU; u++) {
                    if (!x && nz) {  // warp-uniform refill from the next non-zero word of the row
                        const int src = __ffs(nz) - 1;
                        nz &= nz - 1;
                        x = __shfl_sync(0xffffffffu, bw, src);
                        kb = (w0 + (uint32_t)src) * 32u;
                    }
                    k[u] = 0xFFFFFFFFu;
                    if (x) {
                        k[u] = kb + (uint32_t)(__ffs(x) - 1);
                        x &= x - 1;
                    }
                }
                uint32_t cw[kSplitU];
#pragma unroll
                for (int u = 0; u < kSplitU; u++) cw[u] = k[u] != 0xFFFFFFFFu ? __ldcg(TC + (uint64_t)k[u] * W) : 0u;
                uint32_t lb[kSplitU], lc[kSplitU];
                unsigned take = 0;  // bit u: (i, k[u]) in T_B and (k[u], j) in T_C for this lane's j
#pragma unroll
                for (int u = 0; u < kSplitU; u++) {
                    lb[u] = lc[u] = 0u;
                    if (mine && ((cw[u] >> lane) & 1u)) {
                        take |= 1u << u;
                        lb[u] = __ldcg(LB + k[u]);
                        lc[u] = __ldcg(LC + (uint64_t)k[u] * np);
                    }
                }
                hits += (unsigned)__popc(take);
#pragma unroll
                for (int u = 0; u < kSplitU; u++)
                    if ((take >> u) & 1u) {
                        const unsigned long long cand = (unsigned long long)lb[u] + lc[u];
                        best = cand < best ? cand : best;
                    }
            }
        }
    }
    *splits += hits;
    return best;
}

// One block (4 warps) per (non-terminal A, row word of 32 rows): every new pair of A in those
// rows (the bits of N_A, before the Jacobi merge) gets its length. A warp takes 32 words of a
// flagged row at a time and, for each non-zero word, the up to 32 pairs in it.
__global__ void __launch_bounds__(128, 6) k_lengths(const QDesc *qd, uint32_t *L, uint64_t lplane) {
    const QDesc &q = *qd;
    const uint32_t rw = (q.n + 31u) / 32u;
    const int a = (int)(blockIdx.x / rw);
    const uint32_t wq = blockIdx.x % rw;
    const uint32_t parity = (uint32_t)(q.st->iter & 1ull);
    uint32_t rows = __ldcg((parity ? q.R0 : q.R1) + (uint64_t)a * q.W + wq) & rows_in_word(q.n, wq);
    if (!rows) return;
    int r0 = -1, r1 = -1;
    for (int g = 0; g < q.n_groups; g++)
        if (q.rules[q.gstart[g]].lhs == a) {
            r0 = q.gstart[g];
            r1 = q.gstart[g + 1];
        }
    if (r0 < 0) return;
    const uint32_t *N = (parity ? q.X0 : q.X1) + (uint64_t)a * q.plane;
    uint32_t *LA = L + (uint64_t)a * lplane;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t W = q.W;
    unsigned long long splits = 0;
    while (rows) {
        const uint32_t i = wq * 32u + (uint32_t)(__ffs(rows) - 1);
        rows &= rows - 1;
        for (uint32_t w0 = (uint32_t)warp * 32u; w0 < W; w0 += 128u) {
            const uint32_t nw = (w0 + lane < W) ? __ldcg(N + (uint64_t)i * W + w0 + lane) : 0u;
            unsigned nz = __ballot_sync(0xffffffffu, nw != 0u);
            while (nz) {
                const int src = __ffs(nz) - 1;
                nz &= nz - 1;
                const uint32_t bits = __shfl_sync(0xffffffffu, nw, src);
                const uint32_t w = w0 + (uint32_t)src;
                const unsigned long long best = min_split(q, L, lplane, r0, r1, i, w, bits, lane, &splits);
                if ((bits >> lane) & 1u)
                    LA[(uint64_t)i * q.n_pad + w * 32u + lane] = best >= 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)best;
            }
        }
    }
    if (q.profile) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) splits += __shfl_xor_sync(0xffffffffu, splits, o);
        if (lane == 0 && splits) atomicAdd(&q.st->len_splits, splits);
    }
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
    k_seed_lengths<<<blocks, 256, 0, s>>>(c->d_q, c->d_L, c->lplane, eps_mask(c));
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

int lengths_enqueue_iteration(cfpq_ctx *c, cudaStream_t s) {
    const uint32_t blocks = (uint32_t)((uint64_t)c->n_nt * ((c->n + 31) / 32));
    k_lengths<<<blocks, 128, 0, s>>>(c->d_q, c->d_L, c->lplane);
    c->iter_launches++;
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

int lengths_of_triples(cfpq_ctx *c, const cfpq_triple *d_tr, size_t count, uint32_t *d_out, cudaStream_t s) {
    if (count == 0) return CFPQ_OK;
    const uint32_t blocks = (uint32_t)std::min<uint64_t>((count + 255) / 256, 148ull * 32);
    k_triple_lengths<<<blocks, 256, 0, s>>>(d_tr, count, c->d_L, c->lplane, c->n_pad, d_out);
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

}  // namespace cfpq
