// Device-side state and CUDA-core kernels of the CFPQ closure (Algorithm 1, Section 4.2).
//
// Layout in HBM (one query): for every non-terminal A, a bit-packed n_pad x n_pad matrix,
// row-major, 32-bit words, bit j of row i at word i*W + j/32, bit j%32 (W = n_pad/32):
//   T[A]      the current closure T_A
//   X[p][A]   p = 0, 1: the two delta planes; in iteration `it`, X[it&1] holds the pairs
//             added by the previous iteration (D, read by the semi-naive products) and
//             X[(it+1)&1] collects the pairs added now (N)
//   R[p][A]   row bitmaps of X[p][A] (bit i set iff row i of X[p][A] may be non-zero)
//   Trow[A]   row bitmap of T[A] (bit i set iff row i of T[A] is non-empty)
//   TT[A]     T_A transposed, refreshed before tensor-core products that read it
//   occA[A]   tensor path, tile skipping: bit (m-tile, K slice) set iff the 128 x 128-bit tile of
//             T_A is non-zero; occB[A]: bit (n-tile, K slice) set iff the 256 x 128-bit tile of
//             T_A^T is non-zero (the same bits of T_A, tiled as a right operand). SWK words
//             per tile row; refreshed at the start of a loop execution for operands that changed
//   Tsum[A]   word summary of T_A, SW words per row (ceil(W / 32) rounded up to a multiple of
//             4), bit w of row i set iff word w of row i of T_A may be non-zero; kept by every
//             writer of T on the matrix paths (seed, product epilogues, merges) so that a scan
//             of a row of T reads only its non-zero words
//   TTsum[A]  single-path lengths only: the same summary of TT_A (with lengths kept, TT_A is
//             updated pair by pair by the seed and the merge)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cfpq.h"

namespace cfpq {

constexpr int kMaxNT = CFPQ_MAX_NONTERM;

// kErrDevice: a tensor-core product gave up on a bounded wait, so some of its output tiles
// are missing; the loop stops and the solve fails (CFPQ_ERR_CUDA) instead of converging on an
// incomplete product
enum : uint32_t { kErrNone = 0, kErrIterLimit = 1, kErrTimeout = 2, kErrDevice = 3 };

// A loop execution that adds at most kSmallDelta pairs is "small"; after kSwitchAfter small
// executions in a row, a loop that may switch hands the closure to the worklist path (a long
// chain of derivations: one pair per execution would cost a matrix pass per pair).
constexpr unsigned kSmallDelta = 8, kSwitchAfter = 64;

// Per-query device state; one instance in device memory per context.
struct DevState {
    unsigned long long iter;            // loop executions completed
    unsigned long long max_iter;
    unsigned long long deadline_ns;     // %globaltimer deadline, 0 = none
    unsigned long long new_bits;
    unsigned long long seed_bits;
    unsigned long long tensor_products;
    unsigned long long gather_products;
    unsigned int changed;               // set by any product that added a pair this iteration
    unsigned int error;
    unsigned int done;                  // loop ended (converged or error)
    unsigned int cont;                  // loop condition written by the tail
    unsigned int dirty[kMaxNT];         // T[A] changed since TT[A] was rebuilt
    unsigned long long dcount[2][kMaxNT];  // pairs in X[p][A]
    unsigned int use_tensor[kMaxNT];    // per group, 1 = tensor product this iteration (AUTO: chosen per iteration)
    unsigned long long tcount[kMaxNT];  // pairs in T[A] (seed + every product's new pairs)
    unsigned int tt_now[kMaxNT];        // AUTO path: g + 1 if group g refreshes TT[A] this iteration, else 0
    unsigned long long prof_words;      // profile mode: 32-bit words the gather products read or wrote
    unsigned int list_len[2];           // gather items listed for the loop execution of this parity (single-query path)
    unsigned long long useful_macs;     // profile mode: sum over tensor products of nnz(col k of T_B) nnz(row k of T_C)
    unsigned int small_run;             // consecutive executions that added at most kSmallDelta pairs
    unsigned int to_worklist;           // the loop stopped to hand the closure to the worklist path
    unsigned int pad_len;
    unsigned long long len_splits;      // lengths, profile mode: (production, middle node) splits examined
    unsigned int odirty[kMaxNT];        // T[A] changed since its tile occupancy was computed
    unsigned int occ_now[kMaxNT];       // tile occupancy of A to be recomputed at the next tensor execution
    unsigned long long tc_live_steps;   // K steps the tensor-core products issued (after tile skipping)
    unsigned int plan_count[kMaxNT][2]; // tile skipping: live output tiles listed for group g, by execution parity
    unsigned int plan_take[kMaxNT][2];  // tile skipping: listed tiles already claimed by a CTA
    unsigned int occ_probe;             // AUTO: refresh tile occupancy this execution for the cost model
    unsigned long long block_records;   // sharded solve: records packed by the last export
    unsigned int block_bad;             // sharded solve: an imported record was out of range
    unsigned int skip;                  // graph loop: the remaining executions of this unrolled body do nothing
    unsigned int any_next;              // AUTO: the next execution has a tensor product (or an occupancy probe)
    unsigned int tc_diag[6];            // first tensor product that gave up: wait site, CTA + 1, group,
                                        // execution, listed tiles, tiles claimed
    unsigned int loop_launches;         // persistent loop launches of this solve
    unsigned int loop_go;               // persistent loop: the next execution runs in this launch
    unsigned long long loop_execs;      // loop executions those launches ran
    unsigned long long gbar;            // grid barriers of the persistent loop: block arrivals this solve
};

struct Rule {
    int32_t lhs, b, c, pad;
};

// Everything a kernel needs about one query; lives in device memory.
struct QDesc {
    uint32_t n, n_pad, W;
    int32_t n_nt, n_rules, n_groups, schedule, n_unary, n_eps;
    int32_t profile, allow_switch;      // allow_switch: long runs of tiny deltas end the loop (worklist next)
    uint64_t plane;                     // words per matrix = n_pad * W
    uint64_t n_edges;
    uint32_t *T, *TT, *X0, *X1, *R0, *R1, *Trow;
    uint32_t *occA, *occB;              // tile occupancy (NULL: dense tensor products)
    uint32_t *occCA, *occCB;            // per (non-terminal, K slice): m-tiles / n-tiles whose tile is non-zero
    uint32_t *occKnown;                 // per non-terminal: its occupancy (and counts) has been computed
    int32_t tensor_kind;                // CFPQ_TENSOR_FP8 or _FP4 (the product choice's rate)
    uint32_t KS, SWK;                   // K slices of 128 bits per row; occupancy words per tile row
    uint32_t *Tsum;                     // word summary of T (NULL in batched launches)
    uint32_t *TTsum;                    // word summary of TT (NULL unless lengths are kept)
    uint32_t SW;                        // summary words per row (a multiple of 4)
    uint32_t row0, row1;                // rows the products compute: [row0, row1) (0, n_pad: all;
                                        // a sharded solve's row block, multiples of 256)
    const Rule *rules;                  // sorted by lhs; group g = rules[gstart[g] .. gstart[g+1])
    const int32_t *gstart;
    const int2 *nt_rules;               // per non-terminal A: its productions rules[x .. y) (-1, -1: none)
    const int2 *unary;                  // (lhs, term)
    const int32_t *eps;
    const cfpq_edge *edges;
    DevState *st;
};

// Mutable state is read with ld.global.cg (L2, not L1): the persistent batched kernel
// reads, after a grid barrier, words that other SMs wrote in an earlier phase.
__device__ __forceinline__ bool test_bit(const uint32_t *bm, uint32_t i) {
    return (__ldcg(bm + (i >> 5)) >> (i & 31)) & 1u;
}

__device__ __forceinline__ unsigned long long ld_u64(const unsigned long long *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned ld_u32(const unsigned *p) { return __ldcg(p); }

// Rows (of the 32 in row word wq) of a query that has n rows: mask of rows that exist.
__device__ __forceinline__ uint32_t rows_in_word(uint32_t n, uint32_t wq) {
    const uint32_t left = n - wq * 32u;
    return left >= 32u ? 0xFFFFFFFFu : ((1u << left) - 1u);
}

// Rows of row word wq that the query's products compute (its row block [row0, row1), whose
// ends are multiples of 32).
__device__ __forceinline__ uint32_t rows_of_block(const QDesc &q, uint32_t wq) {
    return (wq * 32u >= q.row0 && wq * 32u < q.row1) ? 0xFFFFFFFFu : 0u;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier of a persistent launch whose blocks are all resident (a cooperative launch):
// every thread of every block calls it. st->gbar counts the blocks' arrivals over the solve;
// a launch's barriers complete at base + k gridDim.x (k = 1, 2, ...), and target (shared
// memory, set by grid_sync_start) is the block's next one. The writes before the barrier are
// visible to every block after it: each block's writes are ordered before its arrival (block
// barrier, then a device-scope fence), and its loads after the release (a device-scope fence
// after the count reached the target, then a block barrier). A block that waits longer than
// kGridWaitNs, or sees kErrDevice, records kErrDevice and returns false. The limit is far
// above any one loop phase (one execution's gathers at most: a phase this long means a
// closure that no timeout of the caller would let finish); it bounds a wait on blocks that
// never arrive, which the cooperative launch rules out.
constexpr unsigned long long kGridWaitNs = 300ull * 1000 * 1000 * 1000;
__device__ inline void grid_sync_start(DevState *st, unsigned long long &target) {
    if (threadIdx.x == 0) {
        // fewer than gridDim.x arrivals can precede this read: the first barrier needs every block
        const unsigned long long c = ld_u64(&st->gbar);
        target = c - c % gridDim.x + gridDim.x;
    }
    __syncthreads();
}
__device__ inline bool grid_sync(DevState *st, unsigned long long &target) {
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned ok = 1u;
        const unsigned long long t = target;
        __threadfence();
        atomicAdd(&st->gbar, 1ull);
        const unsigned long long t0 = globaltimer_ns();
        for (unsigned spin = 0; ld_u64(&st->gbar) < t; spin++) {
            if ((spin & 31u) == 31u &&
                (ld_u32(&st->error) == kErrDevice || globaltimer_ns() - t0 > kGridWaitNs)) {
                ok = 0u;
                atomicExch(&st->error, kErrDevice);
                break;
            }
        }
        __threadfence();
        target = t + gridDim.x;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0u;
}

// ------------------------------------------------------------------------------------
// Matrix initialisation (Algorithm 1, before the loop): T_ij gets {A | A -> x} for each
// edge (i, x, j); A -> eps adds (m, m). Every seeded pair is also a delta pair of
// iteration 0 so that the first semi-naive iteration joins everything with everything.
// ------------------------------------------------------------------------------------
// block_cnt (shared memory, one counter per non-terminal) gathers the new pairs of a block for
// one global update per non-terminal; NULL: a global atomic per new pair.
__device__ __forceinline__ void seed_pair(const QDesc &q, int a, uint32_t i, uint32_t j,
                                          unsigned long long *cnt, unsigned *block_cnt = nullptr) {
    const uint64_t w = (uint64_t)a * q.plane + (uint64_t)i * q.W + (j >> 5);
    const uint32_t bit = 1u << (j & 31);
    const uint32_t old = atomicOr(&q.T[w], bit);
    if (!(old & bit)) {
        atomicOr(&q.X0[w], bit);
        atomicOr(&q.R0[(uint64_t)a * q.W + (i >> 5)], 1u << (i & 31));
        atomicOr(&q.Trow[(uint64_t)a * q.W + (i >> 5)], 1u << (i & 31));
        if (block_cnt) {
            atomicAdd(&block_cnt[a], 1u);
        } else {
            atomicAdd(&q.st->dcount[0][a], 1ull);
            atomicAdd(&q.st->tcount[a], 1ull);
        }
        if (q.Tsum) atomicOr(&q.Tsum[((uint64_t)a * q.n_pad + i) * q.SW + (j >> 10)], 1u << ((j >> 5) & 31));
        if (q.TTsum) {
            atomicOr(&q.TT[(uint64_t)a * q.plane + (uint64_t)j * q.W + (i >> 5)], 1u << (i & 31));
            atomicOr(&q.TTsum[((uint64_t)a * q.n_pad + j) * q.SW + (i >> 10)], 1u << ((i >> 5) & 31));
        }
        (*cnt)++;
    }
}

// Every thread of the block calls this (the per-non-terminal counts are gathered per block).
__device__ inline void seed_query(const QDesc &q, uint64_t tid, uint64_t nthreads) {
    __shared__ unsigned s_cnt[kMaxNT];
    for (int a = threadIdx.x; a < q.n_nt; a += blockDim.x) s_cnt[a] = 0u;
    __syncthreads();
    unsigned long long cnt = 0;
    for (uint64_t e = tid; e < q.n_edges; e += nthreads) {
        const cfpq_edge ed = q.edges[e];
        for (int u = 0; u < q.n_unary; u++)
            if (q.unary[u].y == ed.label) seed_pair(q, q.unary[u].x, ed.src, ed.dst, &cnt, s_cnt);
    }
    for (uint64_t t = tid; t < (uint64_t)q.n_eps * q.n; t += nthreads) {
        const int a = q.eps[t / q.n];
        const uint32_t m = (uint32_t)(t % q.n);
        seed_pair(q, a, m, m, &cnt, s_cnt);
    }
    (void)cnt;  // the block's new pairs are the sum of s_cnt
    __syncthreads();
    for (int a = threadIdx.x; a < q.n_nt; a += blockDim.x)
        if (s_cnt[a]) {
            atomicAdd(&q.st->dcount[0][a], (unsigned long long)s_cnt[a]);
            atomicAdd(&q.st->tcount[a], (unsigned long long)s_cnt[a]);
        }
    if (threadIdx.x == 0) {  // one update of the seed total per block, not one per thread
        unsigned long long total = 0;
        for (int a = 0; a < q.n_nt; a++) total += s_cnt[a];
        if (total) atomicAdd(&q.st->seed_bits, total);
    }
}

// ------------------------------------------------------------------------------------
// Semi-naive bit-gather product for all productions with one left-hand side A:
//   N_A |= (D_B x T_C  u  T_B x D_C) \ T_A      for every A -> B C
// where D = pairs added by the previous iteration. One warp owns row i of A and a chunk
// of 32*CPL words of that row; it ORs whole rows of the right operand selected by the set
// bits of the left operand's row ("AND" = the bit test, "OR" = the accumulation). The
// OR-merge into T_A and the change detection are fused at the end.
// ------------------------------------------------------------------------------------
// Rows gathered per step: the loads of kGatherU rows are issued before any of them is
// OR-ed in, so a warp keeps kGatherU row reads in flight instead of one.
constexpr int kGatherU = 4;
// 32-word chunks of a left-operand row whose loads are issued together when a row is scanned.
constexpr int kScanChunks = 4;

template <int CPL>
__device__ __forceinline__ void or_rows_for_bits(uint32_t (&acc)[CPL], uint32_t bw, uint32_t w0,
                                                 const uint32_t *__restrict__ rhs_plane, uint32_t W,
                                                 uint32_t base, int lane, unsigned &rows) {
    unsigned nz = __ballot_sync(0xffffffffu, bw != 0);
    rows += __popc(bw);
    uint32_t bits = 0, kb = 0;  // set bits of the current left word (warp-uniform) and its first column
    while (nz || bits) {
        const uint32_t *r[kGatherU];
#pragma unroll
        for (int u = 0; u < kGatherU; u++) {
            if (!bits && nz) {  // warp-uniform: refill from the next non-zero word of the block
                const int src = __ffs(nz) - 1;
                nz &= nz - 1;
                bits = __shfl_sync(0xffffffffu, bw, src);
                kb = (w0 + src) * 32u;
            }
            r[u] = nullptr;
            if (bits) {
                const uint32_t k = kb + (uint32_t)(__ffs(bits) - 1);
                bits &= bits - 1;
                r[u] = rhs_plane + (uint64_t)k * W + base;
            }
        }
        uint32_t v[kGatherU][CPL];
#pragma unroll
        for (int u = 0; u < kGatherU; u++)
#pragma unroll
            for (int c = 0; c < CPL; c++) {
                const uint32_t col = base + lane + 32 * c;
                v[u][c] = (r[u] && col < W) ? __ldcg(r[u] + lane + 32 * c) : 0u;
            }
#pragma unroll
        for (int u = 0; u < kGatherU; u++)
#pragma unroll
            for (int c = 0; c < CPL; c++) acc[c] |= v[u][c];
    }
}

// blk_new != NULL: the new pairs are added to blk_new[A] (the calling block's shared table,
// which the caller flushes into the counts and flags once per block); NULL: straight into the
// device-side counts and flags.
// WRITE_CHUNK: the chunk of row i of N_A is written whole (its new bits, zeros elsewhere)
// instead of ORed into, so N need not be cleared first. Valid where every product is a gather
// and every chunk of a listed row is listed (the grouped launch): a row whose delta bit is set
// is then entirely this execution's, and no other row of N is read before it is rewritten.
template <int CPL, bool WRITE_CHUNK = false>
__device__ inline void gather_row_chunk(const QDesc &q, int g, uint32_t i, uint32_t ch, int lane,
                                        uint32_t parity, unsigned long long *blk_new = nullptr) {
    const uint32_t W = q.W;
    const uint64_t plane = q.plane;
    const uint32_t *D = parity ? q.X1 : q.X0;
    uint32_t *N = parity ? q.X0 : q.X1;
    const uint32_t *DR = parity ? q.R1 : q.R0;
    uint32_t *NR = parity ? q.R0 : q.R1;
    const DevState *st = q.st;
    const uint32_t base = ch * 32u * CPL;
    const int r0 = q.gstart[g], r1 = q.gstart[g + 1];
    const int A = q.rules[r0].lhs;

    uint32_t acc[CPL];
#pragma unroll
    for (int c = 0; c < CPL; c++) acc[c] = 0;
    bool touched = false;
    unsigned rows = 0, scans = 0;  // gathered rows (this lane's share), scanned row words

    for (int r = r0; r < r1; r++) {
        const int B = q.rules[r].b, C = q.rules[r].c;
        // D_B x T_C: row i of the left delta selects rows of the full right operand
        if (test_bit(DR + (uint64_t)B * W, i)) {
            touched = true;
            scans += W;
            const uint32_t *rowB = D + (uint64_t)B * plane + (uint64_t)i * W;
            for (uint32_t w0 = 0; w0 < W; w0 += 32 * kScanChunks) {
                uint32_t bw[kScanChunks];  // the chunks' loads are issued together
#pragma unroll
                for (int u = 0; u < kScanChunks; u++) {
                    const uint32_t w = w0 + 32u * u + lane;
                    bw[u] = w < W ? __ldcg(rowB + w) : 0u;
                }
#pragma unroll
                for (int u = 0; u < kScanChunks; u++)
                    or_rows_for_bits<CPL>(acc, bw[u], w0 + 32u * u, q.T + (uint64_t)C * plane, W, base, lane, rows);
            }
        }
        // T_B x D_C: only rows k of the right delta that may be non-zero
        if (ld_u64(&st->dcount[parity][C]) != 0 && test_bit(q.Trow + (uint64_t)B * W, i)) {
            touched = true;
            const uint32_t *rowB = q.T + (uint64_t)B * plane + (uint64_t)i * W;
            const uint32_t *rC = DR + (uint64_t)C * W;
            if (q.Tsum) {
                // only the words of row i of T_B that its word summary flags
                const uint32_t *sumB = q.Tsum + ((uint64_t)B * q.n_pad + i) * q.SW;
                scans += q.SW;
                for (uint32_t s0 = 0; s0 < q.SW; s0 += 32) {
                    const uint32_t sv = (s0 + lane < q.SW) ? __ldcg(sumB + s0 + lane) : 0u;
                    unsigned snz = __ballot_sync(0xffffffffu, sv != 0u);
                    while (snz) {
                        const int src = __ffs(snz) - 1;
                        snz &= snz - 1;
                        const uint32_t flagged = __shfl_sync(0xffffffffu, sv, src);
                        const uint32_t w0 = (s0 + (uint32_t)src) * 32u;
                        scans += 2u * (uint32_t)__popc(flagged);
                        const uint32_t bw =
                            ((flagged >> lane) & 1u) ? (__ldcg(rowB + w0 + lane) & __ldcg(rC + w0 + lane)) : 0u;
                        or_rows_for_bits<CPL>(acc, bw, w0, D + (uint64_t)C * plane, W, base, lane, rows);
                    }
                }
                continue;
            }
            scans += 2 * W;
            for (uint32_t w0 = 0; w0 < W; w0 += 32 * kScanChunks) {
                uint32_t bw[kScanChunks];
#pragma unroll
                for (int u = 0; u < kScanChunks; u++) {
                    const uint32_t w = w0 + 32u * u + lane;
                    bw[u] = w < W ? (__ldcg(rowB + w) & __ldcg(rC + w)) : 0u;
                }
#pragma unroll
                for (int u = 0; u < kScanChunks; u++)
                    or_rows_for_bits<CPL>(acc, bw[u], w0 + 32u * u, D + (uint64_t)C * plane, W, base, lane, rows);
            }
        }
    }
    if (!touched) return;

    // fused epilogue: new = acc & ~T_A; merge (in place) and record the delta
    uint32_t *TA = q.T + (uint64_t)A * plane + (uint64_t)i * W;
    uint32_t *NA = N + (uint64_t)A * plane + (uint64_t)i * W;
    const bool inplace = q.schedule == CFPQ_SCHED_INPLACE;
    unsigned cnt = 0;
#pragma unroll
    for (int c = 0; c < CPL; c++) {
        const uint32_t col = base + lane + 32 * c;
        uint32_t nw = 0;
        if (col < W && acc[c]) {
            const uint32_t old = __ldcg(TA + col);
            nw = acc[c] & ~old;
            if (nw) {
                cnt += __popc(nw);
                if (inplace) TA[col] = old | nw;
                if (!WRITE_CHUNK) NA[col] = __ldcg(NA + col) | nw;
            }
        }
        if (WRITE_CHUNK && col < W) NA[col] = nw;
        if (inplace && q.Tsum) {  // the 32 lanes' words form one word of the summary of T_A
            const unsigned sb = __ballot_sync(0xffffffffu, nw != 0u);
            if (lane == 0 && sb) atomicOr(&q.Tsum[((uint64_t)A * q.n_pad + i) * q.SW + ((base + 32u * c) >> 5)], sb);
        }
    }
    const unsigned any = __ballot_sync(0xffffffffu, cnt != 0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (q.profile) {
        // words of this chunk: scanned operand rows, gathered row chunks, T_A chunk read
        // and (when pairs were added) T_A and N_A chunks written
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rows += __shfl_xor_sync(0xffffffffu, rows, o);
        const uint32_t cw = min(32u * CPL, W - base);
        if (lane == 0)
            atomicAdd(&q.st->prof_words, (unsigned long long)scans + (unsigned long long)rows * cw +
                                             (unsigned long long)cw * (any ? 3ull : 1ull));
    }
    if (any && lane == 0) {
        atomicOr(&NR[(uint64_t)A * W + (i >> 5)], 1u << (i & 31));
        if (inplace) atomicOr(&q.Trow[(uint64_t)A * W + (i >> 5)], 1u << (i & 31));
        if (blk_new) {
            atomicAdd(&blk_new[A], (unsigned long long)cnt);
        } else {
            atomicAdd(&q.st->dcount[parity ^ 1u][A], (unsigned long long)cnt);
            atomicAdd(&q.st->tcount[A], (unsigned long long)cnt);
            atomicAdd(&q.st->new_bits, (unsigned long long)cnt);
            q.st->changed = 1u;
            q.st->dirty[A] = 1u;
            q.st->odirty[A] = 1u;
        }
    }
}

// Jacobi schedule: T |= N after all products of the iteration (T_{k+1} = T_k u T_k x T_k).
__device__ inline void merge_row(const QDesc &q, int a, uint32_t i, int lane, uint32_t parity) {
    const uint32_t *N = parity ? q.X0 : q.X1;
    const uint32_t *NR = parity ? q.R0 : q.R1;
    const uint32_t W = q.W;
    if (!test_bit(NR + (uint64_t)a * W, i)) return;
    uint32_t *TA = q.T + (uint64_t)a * q.plane + (uint64_t)i * W;
    const uint32_t *NA = N + (uint64_t)a * q.plane + (uint64_t)i * W;
    for (uint32_t w = lane; w < W; w += 32) TA[w] = __ldcg(TA + w) | __ldcg(NA + w);
    if (lane == 0) atomicOr(&q.Trow[(uint64_t)a * W + (i >> 5)], 1u << (i & 31));
}

// Zeroes the rows of the delta plane that was read this iteration (it becomes N next).
__device__ inline void clear_row(const QDesc &q, int a, uint32_t i, int lane, uint32_t parity) {
    uint32_t *D = parity ? q.X1 : q.X0;
    const uint32_t *DR = parity ? q.R1 : q.R0;
    const uint32_t W = q.W;
    if (!test_bit(DR + (uint64_t)a * W, i)) return;
    uint32_t *row = D + (uint64_t)a * q.plane + (uint64_t)i * W;
    for (uint32_t w = lane; w < W; w += 32) row[w] = 0u;
}

// End of one loop execution (every thread of one block calls it; the block has at least
// max(n_nt, n_groups) threads): clears the old delta's row bitmaps (unless the caller clears
// them later, together with the rows they flag), counts the iteration and decides whether the
// loop continues. The per-non-terminal and per-group bookkeeping is spread over the threads
// (each is a load or a store of its own); thread 0 then takes the decision. Returns the loop
// condition in every thread.
__device__ inline unsigned tail_query(const QDesc &q, int tid, int nthreads, bool zero_read_bitmap) {
    __shared__ unsigned long long s_added;
    __shared__ unsigned s_anytc, s_cont;
    DevState *st = q.st;
    const unsigned long long it = ld_u64(&st->iter);
    const uint32_t old = (uint32_t)(it & 1ull);
    // thread 0's inputs to the decision, loaded together (the products that set changed or
    // error have finished; the others change only here)
    unsigned changed0 = 0u, error0 = 0u, small0 = 0u;
    unsigned long long max_iter0 = 0ull, deadline0 = 0ull;
    if (tid == 0) {
        changed0 = ld_u32(&st->changed);
        error0 = ld_u32(&st->error);
        small0 = ld_u32(&st->small_run);
        max_iter0 = ld_u64(&st->max_iter);
        deadline0 = ld_u64(&st->deadline_ns);
    }
    if (zero_read_bitmap) {
        uint32_t *DR = old ? q.R1 : q.R0;
        for (uint64_t w = tid; w < (uint64_t)q.n_nt * q.W; w += nthreads) DR[w] = 0u;
    }
    if (tid == 0) {
        s_added = 0ull;
        s_anytc = 0u;
    }
    __syncthreads();
    if (tid < q.n_nt) {
        // pairs added now: both parities' counts are loaded (not one after the iteration number)
        const unsigned long long d0 = ld_u64(&st->dcount[0][tid]), d1 = ld_u64(&st->dcount[1][tid]);
        const unsigned long long add = old ? d0 : d1;
        if (add) atomicAdd(&s_added, add);
        st->dcount[old][tid] = 0ull;
    }
    if (tid < q.n_groups && ld_u32(&st->use_tensor[tid])) atomicOr(&s_anytc, 1u);
    __syncthreads();
    if (q.occA) {
        // tile occupancy to refresh at the next tensor execution: what changed now, plus what
        // is still pending if no tensor product ran in this execution
        if (tid < q.n_nt) {
            const unsigned d = ld_u32(&st->odirty[tid]);
            st->odirty[tid] = 0u;
            st->occ_now[tid] = s_anytc ? d : (ld_u32(&st->occ_now[tid]) | d);
        }
        if (tid < q.n_groups) {  // next execution's slots
            st->plan_count[tid][(it + 1ull) & 1ull] = 0u;
            st->plan_take[tid][(it + 1ull) & 1ull] = 0u;
        }
    }
    if (tid == 0) {
        st->list_len[old] = 0u;  // consumed; the next list of this parity is built one execution later
        st->changed = 0u;
        st->iter = it + 1;
        unsigned cont = changed0 ? 1u : 0u;
        if (error0 == kErrDevice) cont = 0;
        if (cont && q.allow_switch) {
            const unsigned run = s_added <= kSmallDelta ? small0 + 1u : 0u;
            st->small_run = run;
            if (run >= kSwitchAfter) {
                st->to_worklist = 1u;
                cont = 0;
            }
        }
        if (cont && it + 1 >= max_iter0) {
            st->error = kErrIterLimit;
            cont = 0;
        }
        const unsigned long long dl = deadline0;
        if (cont && dl && globaltimer_ns() > dl) {
            st->error = kErrTimeout;
            cont = 0;
        }
        st->cont = cont;
        if (!cont) st->done = 1u;
        s_cont = cont;
    }
    __syncthreads();
    return s_cont;
}

}  // namespace cfpq
