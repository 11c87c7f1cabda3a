// Device code of the single-path lengths (Section 5) shared by the lengths kernels and the
// persistent gather loop: the derivation-step encoding, the length of one new pair, and the
// lengths of every pair one loop execution added.
#pragma once
#include "cfpq_device.cuh"

namespace cfpq {

// Derivation step of a pair (one uint32 per cell beside its length, the "witness"), from
// which cfpq_get_path rebuilds the walk: the empty walk (A -> eps), an edge with its label,
// or production rules[r] with middle node k. Ordered so that a smaller word is preferred.
constexpr uint32_t kWitEps = 0x40000000u;             // (m, m) by A -> eps: length 0
constexpr uint32_t kWitEdge = 0x80000000u;            // | label: an edge (m, label, n), length 1
constexpr uint32_t kWitK = 17;                        // split: (r << 17) | k, r < 8192
constexpr uint32_t kMaxLenRules = 1u << (30 - kWitK);

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

// The lengths of the pairs one loop execution added: every thread of every block of a grid of
// 256-thread blocks (kLenWarps warps) calls it, between the products and the merge. Warp g
// scans the rows (A, i) = g, g + warps, ... of the n_nt x n row space whose bit in the new
// delta's row bitmap is set (its lanes test 32 of those rows at once); the bits of N_A's row i
// are exactly the pairs this execution adds (read before the merge). Each new pair goes into
// the warp's queue in shared memory (every lane still holding bits gives one per round);
// whenever 32 are queued, every lane computes one pair's length, so the lanes stay busy however
// the new pairs are spread over rows and words.
__device__ inline void lengths_of_new_pairs(const QDesc &q, uint32_t *L, uint32_t *Wit, uint64_t lplane) {
    __shared__ uint32_t q_i[kLenWarps][kLenQ], q_j[kLenWarps][kLenQ];
    __shared__ uint8_t q_a[kLenWarps][kLenQ];
    __shared__ int2 grp[kMaxNT];  // productions of each left-hand side: [x, y)
    if (threadIdx.x < (unsigned)q.n_nt) grp[threadIdx.x] = q.nt_rules[threadIdx.x];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t gwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t parity = (uint32_t)(ld_u64(&q.st->iter) & 1ull);  // (L2: the persistent loop's tail moves it)
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

}  // namespace cfpq
