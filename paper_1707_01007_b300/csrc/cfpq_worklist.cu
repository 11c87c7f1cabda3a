// Worklist path (CFPQ_PATH_WORKLIST): the closure of Algorithm 1 (Section 4.2) evaluated
// semi-naively at the finest grain, one new pair at a time, on the GPU.
//
// Algorithm 1 joins the whole matrix with itself each iteration. When every iteration adds
// only a pair or two (long derivation chains, e.g. two cycles sharing a node, where the loop
// runs ~pq times), every loop execution costs kernel launches and full-matrix scans for one
// new bit. Here each newly set pair (A, i, j) is instead joined once with its partners:
//   as the left operand of X -> A C:  every (C, j, k) gives (X, i, k)
//   as the right operand of X -> B A: every (B, k, i) gives (X, k, j)
// A derived pair is set with an atomic OR in T_X; if it was new it is pushed on the stack
// (or, when it is the only new pair, handed to the next step in registers). When the stack
// is empty, T is closed under every production: the same least fixpoint as the matrix loop.
// Partners of non-terminals that no production derives (their relation is exactly the seed)
// come from CSR adjacency built from T by set-up kernels; partners of the others from the bit matrices:
// row j of T_C, and row i of T_B^T (T^T is kept for every derived non-terminal).
//
// Warp 0 of block 0 owns the stack. Batches of general pairs are joined by all 16 warps of
// block 0; chains of single-successor steps are walked 31 steps per ballot, and periodic
// chains (which return to their non-terminal) are computed by binary lifting in rounds that
// span up to 128 blocks of a cooperative launch.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "cfpq_internal.h"

namespace cfpq {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kWlWarps = 16, kWlThreads = 32 * kWlWarps;  // per block; block 0's warp 0 runs the worklist
constexpr int kPcSteps = 64, kPcBatch = 16;                 // chain steps per thread and round
constexpr uint32_t kPcBlockSteps = kWlThreads * kPcSteps;   // 32768 per block and round
constexpr int kMaxPcBlocks = 128;                           // blocks a periodic round can span
constexpr int kLiftLevels = 24;          // powers 2^0 .. 2^23 of a period map (covers 128 x 32768 steps)
static_assert((1ull << (kLiftLevels - 1)) >= (unsigned long long)kMaxPcBlocks * kPcBlockSteps, "power tables");
static_assert(kPcSteps % kPcBatch == 0, "batches");
constexpr unsigned long long kPcRoundWaitNs = 5ull * 1000 * 1000 * 1000;   // a round never takes this long
constexpr unsigned long long kPcIdleWaitNs = 600ull * 1000 * 1000 * 1000;  // helpers' wait for work

// A periodic chain: from a pair of non-terminal a the chain goes a -> a1 -> a (P = 2) or
// a -> a (P = 1), each step moving one coordinate of the pair through the unique-successor
// table of a static relation (row: i -> the only k with (k, i) in the partner, when a is a
// right operand; column: j -> the only k with (j, k), when a is a left operand). Over one
// period the row goes through the map G and the column through H (compositions of the
// period's steps; identity if a coordinate does not move), so the pair after P u + r steps
// is (G^u(i), H^u(j)) followed by the first r steps. Powers G^(2^k), H^(2^k) are tabulated.
struct PChain {
    int32_t P, a1, c0, g_id;      // c0: coordinate of step 0 (0 row, 1 column); g_id: G is identity
    int32_t h_id, pad0, pad1, pad2;
    uint64_t m0;                  // step 0's table in uniq
    uint64_t lg, lh;              // G's and H's power tables in lift (level k at + k n)
};

struct WLDesc {
    const int2 *occ;              // per non-terminal a: (production index, side 0 = left / 1 = right)
    const int32_t *occ_start;     // [n_nt + 1]
    const int32_t *is_static;     // [n_nt]
    const uint64_t *out_base;     // [n_nt] start of a's out-CSR offsets in csr_off (static a only)
    const uint64_t *in_base;      // [n_nt] start of a's in-CSR offsets in csr_off
    const uint32_t *csr_off;      // offsets into csr_col (n + 1 per CSR)
    const uint32_t *csr_col;
    const int32_t *needs_tt;      // [n_nt] keep T^T of a (a dynamic and a left operand somewhere)
    const int4 *chain;            // [n_nt] (1, lhs, left, partner) when a has exactly one operand
                                  // occurrence and its partner is static, else (0, ...)
    const uint64_t *chain_base;   // [n_nt] start of the partner's unique-successor table
    const uint32_t *uniq;         // per static partner and direction: the only k, or 0xFFFFFFFF
    const PChain *pchain;         // [n_nt] periodic chain starting at a (P = 0: none)
    const uint32_t *lift;         // per periodic chain: kLiftLevels tables of n entries for G and H
    struct PcCtl *pcc;            // periodic rounds: task and per-block results (device memory)
    int32_t keep_iter;            // 1: leave the loop count of the matrix loop that ran before
    uint32_t *stack;              // triples (a, i, j)
    uint64_t cap;                 // stack capacity in triples
    unsigned long long *items;    // pairs processed
    unsigned int *overflow;
};

__device__ __forceinline__ bool wl_set(const QDesc &q, const WLDesc &w, int x, uint32_t a, uint32_t b) {
    const uint32_t bit = 1u << (b & 31);
    const uint32_t old = atomicOr(&q.T[(uint64_t)x * q.plane + (uint64_t)a * q.W + (b >> 5)], bit);
    if (old & bit) return false;
    if (w.needs_tt[x]) atomicOr(&q.TT[(uint64_t)x * q.plane + (uint64_t)b * q.W + (a >> 5)], 1u << (a & 31));
    return true;
}

// The only candidate pair derived from (a, i, j) when a has one operand occurrence whose
// partner is static and has exactly one partner pair there (precomputed tables).
__device__ __forceinline__ bool single_successor(const int4 *chain, const uint64_t *cbase, const uint32_t *uniq,
                                                 uint32_t a, uint32_t i, uint32_t j, uint32_t &na, uint32_t &ni,
                                                 uint32_t &nj) {
    const int4 d = chain[a];
    if (!d.x) return false;
    const bool left = d.z != 0;
    const uint32_t k = __ldg(uniq + cbase[a] + (left ? j : i));
    if (k == 0xFFFFFFFFu) return false;
    na = (uint32_t)d.y;
    ni = left ? i : k;
    nj = left ? k : j;
    return true;
}

enum : int32_t { kPcIdle = 0, kPcRun = 1, kPcExit = 2 };

// Periodic rounds across blocks. Block 0's warp 0 (the worklist warp) posts a round: the
// chain, the pair its steps start from, and how many blocks take part; every thread of
// those blocks computes 64 consecutive steps (thread g of the grid: steps 64 g + 1 ..
// 64 g + 64). Blocks 1.. wait for a new round number (one thread polls, bounded); block 0's
// helper warps wait on a block barrier that warp 0 arrives at after posting. Each block
// reports its count of valid and of new steps and its last valid pair; warp 0 waits until
// all blocks of the round have reported (bounded) and decides how to continue.
struct PcCtl {
    unsigned gen, done, helpers_gone, pad;
    int32_t cmd, active;
    uint32_t a, i, j;             // the pair the round's steps start from
    PChain pc;
    uint32_t valid[kMaxPcBlocks], fresh[kMaxPcBlocks];
    uint4 last[kMaxPcBlocks];     // (a, i, j, new) of the block's last valid step
};

__shared__ uint32_t s_valid[kWlWarps], s_fresh[kWlWarps];
__shared__ uint4 s_last[kWlThreads];  // each thread's last pair set (a, i, j, new)
__shared__ int s_cmd;

__device__ __forceinline__ void named_barrier(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kWlThreads) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One thread's share of a round (thread g of the grid: steps 64 g + 1 .. 64 g + 64 from the
// round's pair), then the block's counts and last valid pair into the control block. All
// threads of the block call it.
__device__ void pc_block_round(const QDesc &q, const WLDesc &w, PcCtl *c) {
    // the task, read from L2 (it changes between rounds; the round was posted before the
    // barrier that released this block)
    PChain pc;
    pc.P = __ldcg(&c->pc.P);
    pc.a1 = __ldcg(&c->pc.a1);
    pc.c0 = __ldcg(&c->pc.c0);
    pc.g_id = __ldcg(&c->pc.g_id);
    pc.h_id = __ldcg(&c->pc.h_id);
    pc.m0 = __ldcg(reinterpret_cast<const unsigned long long *>(&c->pc.m0));
    pc.lg = __ldcg(reinterpret_cast<const unsigned long long *>(&c->pc.lg));
    pc.lh = __ldcg(reinterpret_cast<const unsigned long long *>(&c->pc.lh));
    const uint32_t n = q.n, P = (uint32_t)pc.P;
    const uint32_t *LG = w.lift + pc.lg, *LH = w.lift + pc.lh, *M0 = w.uniq + pc.m0;
    const uint32_t a0 = __ldcg(&c->a), a1 = (uint32_t)pc.a1;
    const uint64_t t0 = ((uint64_t)blockIdx.x * kWlThreads + threadIdx.x) * (uint64_t)kPcSteps + 1u;
    const uint64_t u0 = t0 / P;
    uint32_t r = (uint32_t)(t0 % P);
    uint32_t g = __ldcg(&c->i), h = __ldcg(&c->j);
    for (int k = 0; k < kLiftLevels; k++)
        if ((u0 >> k) & 1u) {
            if (!pc.g_id) g = g == kNone ? kNone : __ldg(LG + (uint64_t)k * n + g);
            if (!pc.h_id) h = h == kNone ? kNone : __ldg(LH + (uint64_t)k * n + h);
        }
    uint32_t valid = 0, fresh = 0, la = 0, li = 0, lj = 0, lnew = 0;
#pragma unroll 1
    for (int b = 0; b < kPcSteps / kPcBatch; b++) {
        uint32_t pa[kPcBatch], pi[kPcBatch], pj[kPcBatch], old[kPcBatch];
        bool ok[kPcBatch];
#pragma unroll
        for (int s2 = 0; s2 < kPcBatch; s2++) {
            uint32_t xi = g, xj = h;
            if (r == 1u) {
                if (pc.c0 == 0) xi = xi == kNone ? kNone : __ldg(M0 + xi);
                else xj = xj == kNone ? kNone : __ldg(M0 + xj);
            }
            ok[s2] = xi != kNone && xj != kNone;
            pa[s2] = r == 0u ? a0 : a1;
            pi[s2] = xi;
            pj[s2] = xj;
            if (++r == P) {
                r = 0;
                if (!pc.g_id) g = g == kNone ? kNone : __ldg(LG + g);
                if (!pc.h_id) h = h == kNone ? kNone : __ldg(LH + h);
            }
        }
#pragma unroll
        for (int s2 = 0; s2 < kPcBatch; s2++)
            old[s2] = ok[s2] ? atomicOr(&q.T[(uint64_t)pa[s2] * q.plane + (uint64_t)pi[s2] * q.W + (pj[s2] >> 5)],
                                        1u << (pj[s2] & 31))
                             : 0u;
#pragma unroll
        for (int s2 = 0; s2 < kPcBatch; s2++) {
            if (!ok[s2]) continue;
            valid++;
            const bool nw = !((old[s2] >> (pj[s2] & 31)) & 1u);
            if (nw) {
                fresh++;
                if (w.needs_tt[pa[s2]])
                    atomicOr(&q.TT[(uint64_t)pa[s2] * q.plane + (uint64_t)pj[s2] * q.W + (pi[s2] >> 5)],
                             1u << (pi[s2] & 31));
            }
            la = pa[s2];
            li = pi[s2];
            lj = pj[s2];
            lnew = nw ? 1u : 0u;
        }
    }
    s_last[threadIdx.x] = make_uint4(la, li, lj, lnew);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        valid += __shfl_xor_sync(0xffffffffu, valid, o);
        fresh += __shfl_xor_sync(0xffffffffu, fresh, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_valid[threadIdx.x >> 5] = valid;
        s_fresh[threadIdx.x >> 5] = fresh;
    }
    named_barrier(2);
    if (threadIdx.x == 0) {
        uint32_t bv = 0, bf = 0;
        for (int k = 0; k < kWlWarps; k++) {
            bv += s_valid[k];
            bf += s_fresh[k];
        }
        c->valid[blockIdx.x] = bv;
        c->fresh[blockIdx.x] = bf;
        c->last[blockIdx.x] = bv ? s_last[(bv - 1u) / kPcSteps] : make_uint4(0, 0, 0, 0);
        __threadfence();
        atomicAdd(&c->done, 1u);
    }
}

// Stack push of the new pairs of a ballot m (lane l holds pair (x, a, b) if bit l is set).
// With handoff, the first new pair of the join is kept in (ha, hi, hj) instead of pushed.
// shared_top: when set, stack slots are reserved with an atomic on it (several warps push
// at once); otherwise the warp's own top is used.
__device__ __forceinline__ void push_new(const WLDesc &w, unsigned m, uint32_t x, uint32_t a, uint32_t b,
                                         unsigned long long &top, unsigned long long *shared_top, bool handoff,
                                         uint32_t &n_new, uint32_t &ha, uint32_t &hi, uint32_t &hj, int lane) {
    if (!m) return;
    unsigned push = m;
    if (handoff && n_new == 0) {
        const int first = __ffs(m) - 1;
        ha = x;
        hi = __shfl_sync(0xffffffffu, a, first);
        hj = __shfl_sync(0xffffffffu, b, first);
        push = m & (m - 1);
    }
    if (push) {
        const unsigned cnt = __popc(push);
        unsigned long long base = top;
        if (shared_top) {
            if (lane == 0) base = atomicAdd(shared_top, (unsigned long long)cnt);
            base = __shfl_sync(0xffffffffu, base, 0);
        } else {
            top += cnt;
        }
        if ((push >> lane) & 1u) {
            const unsigned long long pos = base + __popc(push & ((1u << lane) - 1u));
            if (pos < w.cap) {
                w.stack[3 * pos] = x;
                w.stack[3 * pos + 1] = a;
                w.stack[3 * pos + 2] = b;
            }
        }
    }
    n_new += __popc(m);
}

// The general join of one popped pair (ca, ci, cj) by the calling warp: through every occurrence of
// ca as an operand, with the partner's CSR (static partner) or bit rows (dynamic partner).
// Returns the number of new pairs.
__device__ uint32_t general_join(const QDesc &q, const WLDesc &w, uint32_t ca, uint32_t ci, uint32_t cj,
                                 unsigned long long &top, unsigned long long *shared_top, bool handoff, uint32_t &ha,
                                 uint32_t &hi, uint32_t &hj, int lane) {
    uint32_t n_new = 0;
    for (int o = w.occ_start[ca]; o < w.occ_start[ca + 1]; o++) {
        const int2 oc = w.occ[o];
        const Rule r = q.rules[oc.x];
        const int x = r.lhs;
        const bool left = oc.y == 0;
        const int p = left ? r.c : r.b;        // partner non-terminal
        const uint32_t key = left ? cj : ci;   // row of T_p (left) or of T_p^T (right)
        if (w.is_static[p]) {
            const uint64_t base = left ? w.out_base[p] : w.in_base[p];
            const uint32_t lo = __ldg(w.csr_off + base + key), hi_ = __ldg(w.csr_off + base + key + 1);
            for (uint32_t e0 = lo; e0 < hi_; e0 += 32) {
                const uint32_t e = e0 + lane;
                bool nw = false;
                uint32_t a = 0, b = 0;
                if (e < hi_) {
                    const uint32_t k = __ldg(w.csr_col + e);
                    a = left ? ci : k;
                    b = left ? k : cj;
                    nw = wl_set(q, w, x, a, b);
                }
                push_new(w, __ballot_sync(0xffffffffu, nw), (uint32_t)x, a, b, top, shared_top, handoff, n_new, ha,
                         hi, hj, lane);
            }
        } else {
            const uint32_t *row = left ? q.T + (uint64_t)p * q.plane + (uint64_t)key * q.W
                                       : q.TT + (uint64_t)p * q.plane + (uint64_t)key * q.W;
            uint32_t *dst_row = q.T + (uint64_t)x * q.plane + (uint64_t)ci * q.W;
            uint32_t *dst_col = q.TT + (uint64_t)x * q.plane + (uint64_t)cj * q.W;  // column cj of T_x
            for (uint32_t w0 = 0; w0 < q.W; w0 += 32) {
                uint32_t bits = (w0 + lane < q.W) ? __ldcg(row + w0 + lane) : 0u;
                if (!left && bits) {
                    // the derived pairs (x, k, cj) fill column cj of T_x: one word-wide OR
                    // into T_x^T per 32 of them; the ones not there yet are then set in T_x,
                    // and a pair is new where its bit of T_x was clear. T_x decides, as for
                    // every other way of setting a pair: a pair set at the same time through
                    // T_x first (wl_set, then T_x^T) would otherwise count once on each side
                    const uint32_t old = atomicOr(dst_col + w0 + lane, bits);
                    bits &= ~old;
                    for (uint32_t nb = bits; nb; nb &= nb - 1) {
                        const uint32_t bk = nb & (0u - nb);
                        const uint32_t k = (w0 + lane) * 32u + (uint32_t)(__ffs(nb) - 1);
                        const uint32_t cbit = 1u << (cj & 31);
                        if (atomicOr(&q.T[(uint64_t)x * q.plane + (uint64_t)k * q.W + (cj >> 5)], cbit) & cbit)
                            bits &= ~bk;
                    }
                }
                if (left && bits) {
                    // the derived pairs (x, ci, k) fill row ci of T_x: one word-wide OR
                    // per 32 of them, and only the bits that were not set yet go on
                    const uint32_t old = atomicOr(dst_row + w0 + lane, bits);
                    bits &= ~old;
                    if (bits && w.needs_tt[x]) {
                        for (uint32_t nb = bits; nb; nb &= nb - 1) {
                            const uint32_t k = (w0 + lane) * 32u + (uint32_t)(__ffs(nb) - 1);
                            atomicOr(&q.TT[(uint64_t)x * q.plane + (uint64_t)k * q.W + (ci >> 5)], 1u << (ci & 31));
                        }
                    }
                }
                while (__any_sync(0xffffffffu, bits != 0)) {
                    bool nw = false;
                    uint32_t a = 0, b = 0;
                    if (bits) {
                        const uint32_t k = (w0 + lane) * 32u + (uint32_t)(__ffs(bits) - 1);
                        bits &= bits - 1;
                        a = left ? ci : k;
                        b = left ? k : cj;
                        nw = true;  // set above, and new
                    }
                    push_new(w, __ballot_sync(0xffffffffu, nw), (uint32_t)x, a, b, top, shared_top, handoff,
                             n_new, ha, hi, hj, lane);
                }
            }
        }
    }
    return n_new;
}

enum : int32_t { kBlkExit = 0, kBlkRound = 1, kBlkJoin = 2 };
constexpr uint32_t kJoinBatch = 64;  // general items joined together by block 0's 16 warps
__shared__ uint4 s_batch[kJoinBatch];
__shared__ uint32_t s_nbatch;
__shared__ unsigned long long s_top;
__shared__ int s_block_cmd;

// A batch of general items (posted by warp 0 in s_batch): warp k of block 0 joins items
// k, k + 16, ..; new pairs go on the stack through the shared top.
__device__ void join_batch(const QDesc &q, const WLDesc &w) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t fresh = 0;
    for (uint32_t k = (uint32_t)warp; k < s_nbatch; k += kWlWarps) {
        const uint4 it = s_batch[k];
        unsigned long long unused = 0;
        uint32_t ha, hi, hj;
        fresh += general_join(q, w, it.x, it.y, it.z, unused, &s_top, false, ha, hi, hj, lane);
    }
    if (fresh && lane == 0) atomicAdd(&q.st->new_bits, (unsigned long long)fresh);
}

// Warp 0 processes the stack until it is empty, the deadline passes or it overflows; the
// other warps help with periodic chains.
// Chain lookahead (warp 0 alone): when the current pair has a single successor through static operands,
// the warp follows the chain up to 31 steps ahead (lane l holds step l + 1) and sets all of
// them with one round of atomics. Every pair set in the batch has its successor set in the
// same batch except the last one, so the chain continues from the last pair if it was new
// and stops otherwise: the pairs processed are exactly those the one-at-a-time loop would
// process, and the result is the same least fixpoint.
__global__ void __launch_bounds__(kWlThreads, 1) k_worklist(const QDesc *qd, WLDesc w, unsigned long long top0) {
    const QDesc &q = *qd;
    const int lane = threadIdx.x & 31;
    PcCtl *pcc = w.pcc;
    if (blockIdx.x > 0) {
        // helper block: one share of every round it is asked to take part in
        unsigned seen = 0;
        const unsigned long long dl = ld_u64(&q.st->deadline_ns);
        for (;;) {
            if (threadIdx.x == 0) {
                int cmd = kPcExit;
                const unsigned long long t0 = globaltimer_ns();
                for (;;) {
                    const unsigned gnow = ld_acquire(&pcc->gen);
                    if (gnow != seen) {
                        seen = gnow;
                        cmd = (int)__ldcg(&pcc->cmd);
                        if (cmd == kPcRun && (int)blockIdx.x >= __ldcg(&pcc->active)) cmd = kPcIdle;
                        break;
                    }
                    const unsigned long long now = globaltimer_ns();
                    if (now - t0 > kPcIdleWaitNs || (dl && now > dl)) {
                        atomicExch(&pcc->helpers_gone, 1u);  // rounds continue on block 0 alone
                        break;
                    }
                    __nanosleep(200);
                }
                s_cmd = cmd;
            }
            __syncthreads();
            const int cmd = s_cmd;
            __syncthreads();
            if (cmd == kPcExit) return;
            if (cmd == kPcRun) pc_block_round(q, w, pcc);
        }
    }
    if (threadIdx.x >= 32) {
        // block 0's helper warps: released by warp 0 for a periodic round or a join batch
        for (;;) {
            named_barrier(1);
            const int cmd = s_block_cmd;
            if (cmd == kBlkExit) return;
            if (cmd == kBlkRound) {
                pc_block_round(q, w, pcc);
            } else {
                join_batch(q, w);
                named_barrier(2);
            }
        }
    }
    unsigned long long top = top0, processed = 0;
    uint32_t ca = 0, ci = 0, cj = 0;  // item handed over in registers
    bool have = false, timed_out = false, force_general = false;
    const unsigned long long deadline = ld_u64(&q.st->deadline_ns);
    __shared__ int4 s_chain[kMaxNT];
    __shared__ uint64_t s_cbase[kMaxNT];
    __shared__ PChain s_pc[kMaxNT];
    for (int a = lane; a < q.n_nt; a += 32) {
        s_chain[a] = w.chain[a];
        s_cbase[a] = w.chain_base[a];
        s_pc[a] = w.pchain[a];
    }
    __syncwarp();
    for (;;) {
        if (!have) {
            if (top == 0) break;
            __syncwarp();  // stack entries written by other lanes of this warp
            top--;
            ca = w.stack[3 * top];
            ci = w.stack[3 * top + 1];
            cj = w.stack[3 * top + 2];
        }
        have = false;
        processed++;
        bool skip_fast = force_general;  // the pair ended a chain: general join only
        force_general = false;
        if ((processed & 4095u) == 0 && deadline &&
            __shfl_sync(0xffffffffu, globaltimer_ns() > deadline ? 1 : 0, 0)) {  // one decision for the warp
            if (lane == 0) q.st->error = kErrTimeout;
            break;
        }
        if (!skip_fast && s_pc[ca].P > 0) {
            // periodic chain: rounds of 32768 steps per block over 1, 2, 4, .. blocks (up to
            // the grid), every thread 64 consecutive steps computed from the round's first pair
            // by binary lifting, with 16 atomics in flight; no dependent walk of the chain. A
            // step with no unique successor ends the chain: the last pair set then goes to the
            // general join below (it may have several successors, or none).
            bool handled = false;  // false: (ca, ci, cj) still needs the general join
            int active = 1;
            for (;;) {
                if (__ldcg(&pcc->helpers_gone)) active = 1;
                if (lane == 0) {
                    pcc->pc = s_pc[ca];
                    pcc->a = ca;
                    pcc->i = ci;
                    pcc->j = cj;
                    pcc->cmd = kPcRun;
                    pcc->active = active;
                    pcc->done = 0u;
                    __threadfence();
                    atomicAdd(&pcc->gen, 1u);
                    s_block_cmd = kBlkRound;
                }
                __syncwarp();
                named_barrier(1);          // block 0's helper warps start
                pc_block_round(q, w, pcc); // block 0's share (warp 0 included)
                int ok = 1;
                if (lane == 0) {
                    const unsigned long long t0 = globaltimer_ns();
                    while (ld_acquire(&pcc->done) < (unsigned)active) {
                        if (globaltimer_ns() - t0 > kPcRoundWaitNs) {
                            ok = 0;
                            break;
                        }
                        __nanosleep(100);
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) q.st->error = kErrTimeout;
                    timed_out = true;
                    break;
                }
                unsigned tot_valid = 0, tot_fresh = 0;
                for (int b = lane; b < active; b += 32) {
                    tot_valid += __ldcg(&pcc->valid[b]);
                    tot_fresh += __ldcg(&pcc->fresh[b]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    tot_valid += __shfl_xor_sync(0xffffffffu, tot_valid, o);
                    tot_fresh += __shfl_xor_sync(0xffffffffu, tot_fresh, o);
                }
                processed += tot_valid;
                if (tot_fresh && lane == 0) atomicAdd(&q.st->new_bits, (unsigned long long)tot_fresh);
                if (tot_valid == 0) break;  // (ca, ci, cj) has no unique successor: general join
                // the last pair set: reported by the block of step tot_valid
                const uint4 e = __ldcg(&pcc->last[(tot_valid - 1u) / kPcBlockSteps]);
                const unsigned long long round_steps = (unsigned long long)active * kPcBlockSteps;
                if (tot_valid < round_steps) {
                    handled = true;
                    if (e.w) {
                        ca = e.x;
                        ci = e.y;
                        cj = e.z;
                        have = true;
                        force_general = true;
                    }
                    break;
                }
                if (!e.w) {
                    handled = true;  // the pair was already set: whoever set it continues
                    break;
                }
                const int expired = __shfl_sync(0xffffffffu, (deadline && globaltimer_ns() > deadline) ? 1 : 0, 0);
                if (expired) {
                    if (lane == 0) q.st->error = kErrTimeout;
                    timed_out = true;
                    break;
                }
                ca = e.x;  // continue from the round's last pair, on twice as many blocks
                ci = e.y;
                cj = e.z;
                active = min(2 * active, (int)gridDim.x);
            }
            if (timed_out) break;
            if (handled) continue;
            skip_fast = true;  // fall through with (ca, ci, cj)
        }
        if (!skip_fast) {
            // chain lookahead
            uint32_t xa = ca, xi = ci, xj = cj, ma = 0, mi = 0, mj = 0;
            int len = 0;
            for (; len < 31; len++) {
                uint32_t na, ni, nj;
                if (!single_successor(s_chain, s_cbase, w.uniq, xa, xi, xj, na, ni, nj)) break;
                xa = na; xi = ni; xj = nj;
                if (lane == len) { ma = na; mi = ni; mj = nj; }
            }
            if (len > 0) {
                const bool nw = lane < len ? wl_set(q, w, (int)ma, mi, mj) : false;
                const unsigned m = __ballot_sync(0xffffffffu, nw);
                processed += (unsigned)len - 1u;
                if (m && lane == 0) atomicAdd(&q.st->new_bits, (unsigned long long)__popc(m));
                if ((m >> (len - 1)) & 1u) {  // the last pair was new: continue from it
                    ca = __shfl_sync(0xffffffffu, ma, len - 1);
                    ci = __shfl_sync(0xffffffffu, mi, len - 1);
                    cj = __shfl_sync(0xffffffffu, mj, len - 1);
                    have = true;
                }
                continue;
            }
        }
        uint32_t ha = 0, hi = 0, hj = 0;
        uint32_t n_new = 0;
        {
            // more general items right below on the stack: join them in one batch on all warps
            uint32_t nb = 1;
            if (lane == 0) {
                s_batch[0] = make_uint4(ca, ci, cj, 0);
                while (nb < kJoinBatch && top > 0) {
                    const uint32_t xa = w.stack[3 * (top - 1)];
                    if (s_pc[xa].P > 0 || s_chain[xa].x) break;  // chains stay with this warp
                    top--;
                    s_batch[nb++] = make_uint4(xa, w.stack[3 * top + 1], w.stack[3 * top + 2], 0);
                }
            }
            nb = __shfl_sync(0xffffffffu, nb, 0);
            top = __shfl_sync(0xffffffffu, top, 0);
            if (nb > 1) {
                processed += nb - 1;
                if (lane == 0) {
                    s_nbatch = nb;
                    s_top = top;
                    s_block_cmd = kBlkJoin;
                }
                __syncwarp();
                named_barrier(1);  // block 0's helper warps join the batch too
                join_batch(q, w);
                named_barrier(2);
                top = s_top;
                if (top > w.cap) {
                    if (lane == 0) atomicExch(w.overflow, 1u);
                    break;
                }
                continue;
            }
        }
        n_new = general_join(q, w, ca, ci, cj, top, nullptr, true, ha, hi, hj, lane);
        if (top > w.cap) {
            if (lane == 0) atomicExch(w.overflow, 1u);
            break;
        }
        if (n_new) {
            ca = ha;
            ci = hi;
            cj = hj;
            have = true;
            if (lane == 0) atomicAdd(&q.st->new_bits, (unsigned long long)n_new);
        }
    }
    if (lane == 0) {
        *w.items = processed;
        if (!w.keep_iter) q.st->iter = 1;
        pcc->cmd = kPcExit;
        __threadfence();
        atomicAdd(&pcc->gen, 1u);  // helper blocks leave
        s_block_cmd = kBlkExit;
    }
    __syncwarp();
    named_barrier(1);  // block 0's helper warps see kPcExit and leave
}

// After the walk: the row bitmap of every T_a (extraction visits only non-empty rows), rebuilt
// from the matrix rather than kept with one more atomic per set pair. One warp per row.
__global__ void k_worklist_rows(const QDesc *qd) {
    const QDesc &q = *qd;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (uint64_t)q.n_nt * q.n) return;
    const uint32_t a = (uint32_t)(warp / q.n), i = (uint32_t)(warp % q.n);
    const uint32_t *row = q.T + (uint64_t)a * q.plane + (uint64_t)i * q.W;
    uint32_t any = 0;
    for (uint32_t w0 = 0; w0 < q.W && !__any_sync(0xffffffffu, any != 0); w0 += 32)
        any |= (w0 + lane < q.W) ? __ldcg(row + w0 + lane) : 0u;
    if (__any_sync(0xffffffffu, any != 0) && lane == 0) atomicOr(&q.Trow[(uint64_t)a * q.W + (i >> 5)], 1u << (i & 31));
}

// Hand-over from the matrix loop: every pair of the current delta plane (the pairs the
// loop added last, not yet joined) goes on the stack. One warp per (non-terminal, row).
__global__ void k_worklist_init_delta(const QDesc *qd, WLDesc w, unsigned long long *top) {
    const QDesc &q = *qd;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (uint64_t)q.n_nt * q.n) return;
    const uint32_t a = (uint32_t)(warp / q.n), i = (uint32_t)(warp % q.n);
    const uint32_t par = (uint32_t)(q.st->iter & 1ull);
    if (!test_bit((par ? q.R1 : q.R0) + (uint64_t)a * q.W, i)) return;
    const uint32_t *row = (par ? q.X1 : q.X0) + (uint64_t)a * q.plane + (uint64_t)i * q.W;
    for (uint32_t w0 = 0; w0 < q.W; w0 += 32) {
        uint32_t bits = (w0 + lane < q.W) ? row[w0 + lane] : 0u;
        while (bits) {
            const uint32_t j = (w0 + lane) * 32u + (uint32_t)(__ffs(bits) - 1);
            bits &= bits - 1;
            const unsigned long long pos = atomicAdd(top, 1ull);
            if (pos < w.cap) {
                w.stack[3 * pos] = a;
                w.stack[3 * pos + 1] = i;
                w.stack[3 * pos + 2] = j;
            }
        }
    }
}

// Every seeded pair goes on the stack (and into T^T where kept).
__global__ void k_worklist_init(const QDesc *qd, WLDesc w, unsigned long long *top) {
    const QDesc &q = *qd;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (uint64_t)q.n_nt * q.n) return;
    const uint32_t a = (uint32_t)(warp / q.n), i = (uint32_t)(warp % q.n);
    if (!test_bit(q.Trow + (uint64_t)a * q.W, i)) return;
    const uint32_t *row = q.T + (uint64_t)a * q.plane + (uint64_t)i * q.W;
    for (uint32_t w0 = 0; w0 < q.W; w0 += 32) {
        uint32_t bits = (w0 + lane < q.W) ? row[w0 + lane] : 0u;
        while (bits) {
            const uint32_t j = (w0 + lane) * 32u + (uint32_t)(__ffs(bits) - 1);
            bits &= bits - 1;
            if (w.needs_tt[a]) atomicOr(&q.TT[(uint64_t)a * q.plane + (uint64_t)j * q.W + (i >> 5)], 1u << (i & 31));
            const unsigned long long pos = atomicAdd(top, 1ull);
            if (pos < w.cap) {
                w.stack[3 * pos] = a;
                w.stack[3 * pos + 1] = i;
                w.stack[3 * pos + 2] = j;
            }
        }
    }
}

// ------------------------------------------------------------------ set-up (device tables)
//
// A non-terminal that no production derives keeps exactly its seed, so its relation is read
// from T (and from T^T, its bit transpose) once the seed is in place. Its two CSRs (by row
// and by column), the unique-successor tables and the power tables of the period maps are
// built here by kernels, each launch covering every static relation (grid y), in the places
// the host laid out: CSR ci = 2 r + dir of the r-th static relation (dir 0: by row, from T;
// 1: by column, from T^T) has its n + 1 offsets at csr_off + ci (n + 1) and its
// unique-successor table at uniq + ci n; map m's power tables start at lift + m L n.
struct CsrPlan {
    const uint32_t *T, *TT;      // bit planes
    uint64_t plane;              // words per plane
    const int32_t *statics;      // [n_static] non-terminal of each static relation
    uint32_t n, W;
};

__device__ __forceinline__ const uint32_t *csr_plane(const CsrPlan &p, uint32_t ci) {
    const int32_t a = p.statics[ci >> 1];
    return ((ci & 1u) ? p.TT : p.T) + (uint64_t)a * p.plane;
}

// Row popcounts: off[ci (n + 1) + i] = |row i| for i < n. One warp per row.
__global__ void k_csr_count(CsrPlan p, uint32_t *csr_off) {
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= p.n) return;
    const uint32_t *row = csr_plane(p, blockIdx.y) + warp * p.W;
    uint32_t c = 0;
    for (uint32_t w = lane; w < p.W; w += 32) c += (uint32_t)__popc(__ldcg(row + w));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) csr_off[(uint64_t)blockIdx.y * (p.n + 1) + warp] = c;
}

// The counts become offsets into the one column array shared by every CSR, in place: the
// CSRs in order, each row's offset = the columns of every row before it (earlier CSRs
// included), off[n] of each CSR = its end. One block of 1024 threads, each scanning a
// contiguous run of rows; the 64-bit total goes to *total, which the host checks against the
// 32-bit offset range before any column is written.
__global__ void __launch_bounds__(1024) k_csr_scan(uint32_t *csr_off, uint32_t n, uint32_t n_csr,
                                                   unsigned long long *total) {
    __shared__ unsigned long long part[1024];
    const uint32_t t = threadIdx.x;
    const uint32_t per = (n + 1023u) / 1024u;
    const uint32_t lo = min(n, t * per), hi = min(n, lo + per);
    unsigned long long base = 0;
    for (uint32_t ci = 0; ci < n_csr; ci++) {
        uint32_t *off = csr_off + (uint64_t)ci * (n + 1);
        unsigned long long sum = 0;
        for (uint32_t i = lo; i < hi; i++) sum += off[i];
        part[t] = sum;
        __syncthreads();
        for (uint32_t o = 1; o < 1024; o <<= 1) {
            const unsigned long long v = t >= o ? part[t - o] : 0ull;
            __syncthreads();
            part[t] += v;
            __syncthreads();
        }
        unsigned long long acc = base + part[t] - sum;
        for (uint32_t i = lo; i < hi; i++) {
            const uint32_t c = off[i];
            off[i] = (uint32_t)acc;
            acc += c;
        }
        base += part[1023];
        if (t == 0) off[n] = (uint32_t)base;
        __syncthreads();  // part is rewritten by the next CSR
    }
    if (t == 0) *total = base;
}

// The columns: row i's set bits in ascending order from col[off[i]]. One warp per row; each
// 32-word chunk of the row is placed by a warp prefix sum of its words' popcounts. Then the
// row's unique-successor entry: its only column, or kNone when it has none or several.
__global__ void k_csr_fill(CsrPlan p, const uint32_t *csr_off, uint32_t *col, uint32_t *uniq) {
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= p.n) return;
    const uint32_t ci = blockIdx.y;
    const uint32_t *row = csr_plane(p, ci) + warp * p.W;
    const uint32_t *off = csr_off + (uint64_t)ci * (p.n + 1);
    const uint32_t start = off[warp];
    uint32_t pos = start;
    for (uint32_t w0 = 0; w0 < p.W; w0 += 32) {
        uint32_t bits = (w0 + lane < p.W) ? __ldcg(row + w0 + lane) : 0u;
        const uint32_t c = (uint32_t)__popc(bits);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        uint32_t q = pos + incl - c;
        while (bits) {
            col[q++] = (w0 + lane) * 32u + (uint32_t)(__ffs(bits) - 1);
            bits &= bits - 1;
        }
        pos += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    if (lane == 0) uniq[(uint64_t)ci * p.n + warp] = pos - start == 1u ? col[start] : kNone;
}

// One period of a periodic chain (grid y): G (row) and H (column) start as the identity and go
// through the unique-successor table of each of its P <= 2 steps, on the coordinate that step
// moves; level 0 of the power tables of the maps that move (map index -1: identity, no table).
struct PeriodSteps {
    int32_t P, col0, col1, g_map, h_map, pad;
    uint64_t m0, m1;  // the steps' tables in uniq
};

__global__ void k_period_maps(const uint32_t *uniq, const PeriodSteps *periods, uint32_t n, uint32_t *lift) {
    const uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= n) return;
    const PeriodSteps ps = periods[blockIdx.y];
    uint32_t g = (uint32_t)y, h = (uint32_t)y;
    for (int st = 0; st < ps.P; st++) {
        const uint32_t *M = uniq + (st == 0 ? ps.m0 : ps.m1);
        uint32_t &f = (st == 0 ? ps.col0 : ps.col1) ? h : g;
        f = f == kNone ? kNone : M[f];
    }
    const uint64_t L = (uint64_t)kLiftLevels * n;
    if (ps.g_map >= 0) lift[(uint64_t)ps.g_map * L + y] = g;
    if (ps.h_map >= 0) lift[(uint64_t)ps.h_map * L + y] = h;
}

// Level lv of every map's power table (grid y: the map) from level lv - 1:
// F^(2^lv) = F^(2^(lv-1)) o F^(2^(lv-1)).
__global__ void k_lift_level(uint32_t *lift, uint32_t n, int lv) {
    const uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= n) return;
    const uint32_t *prev = lift + (uint64_t)blockIdx.y * kLiftLevels * n + (uint64_t)(lv - 1) * n;
    const uint32_t v = prev[y];
    lift[(uint64_t)blockIdx.y * kLiftLevels * n + (uint64_t)lv * n + y] = v == kNone ? kNone : prev[v];
}

// ------------------------------------------------------------------------------------ host

struct WorklistState {
    WLDesc d;
    void *arena = nullptr;
    void *cols = nullptr;  // the CSR columns of the static relations
    unsigned long long *d_top = nullptr;
    int blocks = 1;  // grid of the walk: periodic chains use up to kMaxPcBlocks blocks
};

int worklist_setup(cfpq_ctx *c, bool seeded) {
    const auto t_begin = std::chrono::steady_clock::now();
    const int n_nt = c->n_nt;
    const uint32_t n = c->n, W = c->W;
    cudaStream_t s = c->stream;
    std::vector<int32_t> is_static(n_nt, 1), needs_tt(n_nt, 0);
    for (const Rule &r : c->rules) is_static[r.lhs] = 0;
    // T^T is kept for every derived non-terminal: right-operand joins read T_p^T of a dynamic
    // left partner p, and OR word-wide into T_x^T to find which derived pairs are new
    for (int a = 0; a < n_nt; a++) needs_tt[a] = is_static[a] ? 0 : 1;
    // occurrences of each non-terminal as an operand
    std::vector<std::vector<int2>> occ(n_nt);
    for (size_t k = 0; k < c->rules.size(); k++) {
        occ[c->rules[k].b].push_back(make_int2((int)k, 0));
        occ[c->rules[k].c].push_back(make_int2((int)k, 1));
    }
    std::vector<int2> occ_flat;
    std::vector<int32_t> occ_start(n_nt + 1, 0);
    for (int a = 0; a < n_nt; a++) {
        occ_start[a] = (int32_t)occ_flat.size();
        occ_flat.insert(occ_flat.end(), occ[a].begin(), occ[a].end());
    }
    occ_start[n_nt] = (int32_t)occ_flat.size();
    // layout of the tables of static non-terminals: two CSRs (n + 1 offsets each; the columns
    // are counted on the device) and two unique-successor tables (n entries each)
    std::vector<uint64_t> out_base(n_nt, 0), in_base(n_nt, 0), uniq_out_base(n_nt, 0), uniq_in_base(n_nt, 0);
    std::vector<int> statics;
    uint64_t n_off = 0, n_uniq = 0;
    for (int a = 0; a < n_nt; a++)
        if (is_static[a]) {
            statics.push_back(a);
            out_base[a] = n_off;
            in_base[a] = n_off + n + 1;
            n_off += 2ull * (n + 1);
            uniq_out_base[a] = n_uniq;
            uniq_in_base[a] = n_uniq + n;
            n_uniq += 2ull * n;
        }
    std::vector<int4> chain(n_nt, make_int4(0, 0, 0, 0));
    std::vector<uint64_t> chain_base(n_nt, 0);
    for (int a = 0; a < n_nt; a++) {
        if (occ[a].size() != 1) continue;
        const Rule &r = c->rules[occ[a][0].x];
        const bool left = occ[a][0].y == 0;
        const int p = left ? r.c : r.b;
        if (!is_static[p]) continue;
        chain[a] = make_int4(1, r.lhs, left ? 1 : 0, p);
        chain_base[a] = left ? uniq_out_base[p] : uniq_in_base[p];
    }
    // periodic chains (a -> a or a -> a1 -> a through chain steps): the steps of a period and
    // the places of the power tables of its maps G (row) and H (column), where they move
    std::vector<PChain> pchain(n_nt);
    memset(pchain.data(), 0, sizeof(PChain) * n_nt);
    std::vector<PeriodSteps> periods;
    int n_maps = 0;
    for (int a = 0; a < n_nt; a++) {
        if (!chain[a].x) continue;
        const int a1 = chain[a].y;
        int P = 0;
        if (a1 == a) P = 1;
        else if (chain[a1].x && chain[a1].y == a) P = 2;
        if (P == 0) continue;
        PeriodSteps ps;
        memset(&ps, 0, sizeof(ps));
        ps.g_map = ps.h_map = -1;
        ps.P = P;
        ps.col0 = chain[a].z != 0 ? 1 : 0;  // left operand: the column moves
        ps.m0 = chain_base[a];
        ps.col1 = P == 2 && chain[a1].z != 0 ? 1 : 0;
        ps.m1 = P == 2 ? chain_base[a1] : 0;
        const bool row_moves = !ps.col0 || (P == 2 && !ps.col1);
        const bool col_moves = ps.col0 || (P == 2 && ps.col1);
        PChain pc;
        memset(&pc, 0, sizeof(pc));
        pc.P = P;
        pc.a1 = a1;
        pc.c0 = ps.col0;
        pc.m0 = chain_base[a];
        pc.g_id = row_moves ? 0 : 1;
        pc.h_id = col_moves ? 0 : 1;
        if (row_moves) {
            ps.g_map = n_maps++;
            pc.lg = (uint64_t)ps.g_map * kLiftLevels * n;
        }
        if (col_moves) {
            ps.h_map = n_maps++;
            pc.lh = (uint64_t)ps.h_map * kLiftLevels * n;
        }
        pchain[a] = pc;
        periods.push_back(ps);
    }
    const uint64_t n_lift = (uint64_t)n_maps * kLiftLevels * n;
    // device arena (the CSR columns follow once their number is known)
    const uint64_t cap_full = (uint64_t)n_nt * (uint64_t)n * (uint64_t)n;
    const uint64_t cap = std::max<uint64_t>(1024, std::min<uint64_t>(cap_full, 1ull << 27));
    struct Part { void **dst; size_t bytes; };
    WorklistState *ws = new WorklistState();
    WLDesc &d = ws->d;
    memset(&d, 0, sizeof(d));
    unsigned long long *d_total = nullptr;
    int32_t *d_statics = nullptr;
    PeriodSteps *d_periods = nullptr;
    const Part parts[] = {{(void **)&d.occ, occ_flat.size() * sizeof(int2) + 8},
                          {(void **)&d.occ_start, occ_start.size() * 4},
                          {(void **)&d.is_static, (size_t)n_nt * 4},
                          {(void **)&d.out_base, (size_t)n_nt * 8},
                          {(void **)&d.in_base, (size_t)n_nt * 8},
                          {(void **)&d.csr_off, n_off * 4 + 8},
                          {(void **)&d.needs_tt, (size_t)n_nt * 4},
                          {(void **)&d.chain, (size_t)n_nt * sizeof(int4)},
                          {(void **)&d.chain_base, (size_t)n_nt * 8},
                          {(void **)&d.uniq, n_uniq * 4 + 8},
                          {(void **)&d.pchain, (size_t)n_nt * sizeof(PChain)},
                          {(void **)&d.lift, n_lift * 4 + 8},
                          {(void **)&d.pcc, sizeof(PcCtl)},
                          {(void **)&d.stack, cap * 12},
                          {(void **)&d.items, 8},
                          {(void **)&d.overflow, 8},
                          {(void **)&ws->d_top, 8},
                          {(void **)&d_total, 8},
                          {(void **)&d_statics, statics.size() * 4 + 8},
                          {(void **)&d_periods, periods.size() * sizeof(PeriodSteps) + 8}};
    size_t total = 0;
    for (const Part &p : parts) total += (p.bytes + 255) / 256 * 256;
    auto fail = [&](int rc) {
        if (ws->arena) ctx_free(c, ws->arena, s);
        if (ws->cols) ctx_free(c, ws->cols, s);
        delete ws;
        return rc;
    };
    cudaError_t e = ctx_alloc(c, &ws->arena, total, s);
    if (e != cudaSuccess) {
        ws->arena = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? CFPQ_ERR_NOMEM : CFPQ_ERR_CUDA);
    }
    char *ptr = static_cast<char *>(ws->arena);
    for (const Part &p : parts) {
        *p.dst = ptr;
        ptr += (p.bytes + 255) / 256 * 256;
    }
    d.cap = cap;
    bool any_periodic = !periods.empty();
    if (any_periodic) {
        // every block of the grid must be resident at once (cooperative launch)
        int dev = 0, sms = 0, per_sm = 0, coop = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_worklist, kWlThreads, 0) == cudaSuccess) {
            const int fit = std::min(kMaxPcBlocks, sms * std::max(per_sm, 0));
            while (ws->blocks * 2 <= fit) ws->blocks *= 2;
        }
        cudaGetLastError();
    }
    bool ok = true;
    auto up = [&](const void *dst, const void *src, size_t bytes) {
        if (bytes && cudaMemcpyAsync(const_cast<void *>(dst), src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
            ok = false;
    };
    up(d.occ, occ_flat.data(), occ_flat.size() * sizeof(int2));
    up(d.occ_start, occ_start.data(), occ_start.size() * 4);
    up(d.is_static, is_static.data(), (size_t)n_nt * 4);
    up(d.out_base, out_base.data(), (size_t)n_nt * 8);
    up(d.in_base, in_base.data(), (size_t)n_nt * 8);
    up(d.needs_tt, needs_tt.data(), (size_t)n_nt * 4);
    up(d.chain, chain.data(), (size_t)n_nt * sizeof(int4));
    up(d.chain_base, chain_base.data(), (size_t)n_nt * 8);
    up(d.pchain, pchain.data(), (size_t)n_nt * sizeof(PChain));
    up(d_statics, statics.data(), statics.size() * 4);
    up(d_periods, periods.data(), periods.size() * sizeof(PeriodSteps));
    if (!ok) return fail(CFPQ_ERR_CUDA);
    // the static relations: the seed, in T (a context handed over from the matrix loop holds
    // it already: no production writes a static non-terminal), and its transpose in T^T
    // (scratch here: the worklist keeps T^T of derived non-terminals only)
    if (!seeded) {
        const int rc = enqueue_reset_and_seed(c, s);
        if (rc != CFPQ_OK) return fail(rc);
    }
    const uint32_t n_csr = 2u * (uint32_t)statics.size();
    unsigned long long n_col = 0;
    CsrPlan plan;
    plan.T = c->d_T;
    plan.TT = c->d_TT;
    plan.plane = c->plane;
    plan.statics = d_statics;
    plan.n = n;
    plan.W = W;
    const uint32_t row_blocks = (uint32_t)std::max<uint64_t>(1, ((uint64_t)n * 32 + 255) / 256);
    const uint32_t key_blocks = (uint32_t)std::max<uint64_t>(1, ((uint64_t)n + 255) / 256);
    if (n_csr) {
        for (int a : statics)
            if (enqueue_transpose_bits(c, a, s) != CFPQ_OK) return fail(CFPQ_ERR_CUDA);
        k_csr_count<<<dim3(row_blocks, n_csr), 256, 0, s>>>(plan, const_cast<uint32_t *>(d.csr_off));
        k_csr_scan<<<1, 1024, 0, s>>>(const_cast<uint32_t *>(d.csr_off), n, n_csr, d_total);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&n_col, d_total, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(CFPQ_ERR_CUDA);
        if (n_col > 0xFFFFFFFFull) return fail(CFPQ_ERR_NOMEM);  // offsets are 32-bit
    }
    if ((e = ctx_alloc(c, &ws->cols, n_col * 4 + 8, s)) != cudaSuccess) {
        ws->cols = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? CFPQ_ERR_NOMEM : CFPQ_ERR_CUDA);
    }
    d.csr_col = static_cast<uint32_t *>(ws->cols);
    if (n_csr)
        k_csr_fill<<<dim3(row_blocks, n_csr), 256, 0, s>>>(plan, d.csr_off, const_cast<uint32_t *>(d.csr_col),
                                                           const_cast<uint32_t *>(d.uniq));
    if (!periods.empty() && n_maps > 0) {  // every period moves a coordinate: n_maps >= 1
        uint32_t *lift = const_cast<uint32_t *>(d.lift);
        k_period_maps<<<dim3(key_blocks, (uint32_t)periods.size()), 256, 0, s>>>(d.uniq, d_periods, n, lift);
        for (int lv = 1; lv < kLiftLevels; lv++) k_lift_level<<<dim3(key_blocks, (uint32_t)n_maps), 256, 0, s>>>(lift, n, lv);
    }
    // the worklist may run on another stream than the context's
    if (cudaGetLastError() != cudaSuccess || (!c->pooled && cudaStreamSynchronize(s) != cudaSuccess))
        return fail(CFPQ_ERR_CUDA);
    c->h_wl = ws;
    c->stats.worklist_setup_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_begin).count();
    return CFPQ_OK;
}

void worklist_release(cfpq_ctx *c) {
    WorklistState *ws = static_cast<WorklistState *>(c->h_wl);
    if (!ws) return;
    ctx_free(c, ws->arena, c->stream);
    if (ws->cols) ctx_free(c, ws->cols, c->stream);
    delete ws;
    c->h_wl = nullptr;
}

// After enqueue_reset_and_seed: stack the seeds, run the warp, read its counters.
int worklist_run(cfpq_ctx *c, cudaStream_t s, bool from_delta) {
    WorklistState *ws = static_cast<WorklistState *>(c->h_wl);
    if (!ws) return CFPQ_ERR_UNSUPPORTED;
    WLDesc &d = ws->d;
    d.keep_iter = from_delta ? 1 : 0;
    if (cudaMemsetAsync(ws->d_top, 0, 8, s) != cudaSuccess || cudaMemsetAsync(d.overflow, 0, 8, s) != cudaSuccess ||
        cudaMemsetAsync(d.pcc, 0, sizeof(PcCtl), s) != cudaSuccess)
        return CFPQ_ERR_CUDA;
    const uint64_t rows = (uint64_t)c->n_nt * c->n;
    if (from_delta) {
        // T^T of every derived non-terminal from T as the loop left it, then the delta stacked
        if (enqueue_all_transposes(c, s) != CFPQ_OK) return CFPQ_ERR_CUDA;
        k_worklist_init_delta<<<(uint32_t)((rows * 32 + 255) / 256), 256, 0, s>>>(c->d_q, d, ws->d_top);
    } else {
        if (cudaMemsetAsync(c->d_TT, 0, (size_t)c->n_nt * c->plane * 4, s) != cudaSuccess) return CFPQ_ERR_CUDA;
        k_worklist_init<<<(uint32_t)((rows * 32 + 255) / 256), 256, 0, s>>>(c->d_q, d, ws->d_top);
    }
    unsigned long long top = 0;
    if (cudaMemcpyAsync(&top, ws->d_top, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CFPQ_ERR_CUDA;
    if (top > d.cap) return CFPQ_ERR_NOMEM;
    {
        const QDesc *qd = c->d_q;
        void *args[] = {(void *)&qd, (void *)&d, (void *)&top};
        const cudaError_t e = ws->blocks > 1
                                  ? cudaLaunchCooperativeKernel((const void *)k_worklist, dim3(ws->blocks),
                                                                dim3(kWlThreads), args, 0, s)
                                  : cudaLaunchKernel((const void *)k_worklist, dim3(1), dim3(kWlThreads), args, 0, s);
        if (e != cudaSuccess) return CFPQ_ERR_CUDA;
    }
    k_worklist_rows<<<(uint32_t)((rows * 32 + 255) / 256), 256, 0, s>>>(c->d_q);
    c->iter_launches = 1;
    c->fixed_launches += 3;
    unsigned overflow = 0;
    unsigned long long items = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&overflow, d.overflow, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&items, d.items, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CFPQ_ERR_CUDA;
    c->stats.worklist_items = (int64_t)items;
    return overflow ? CFPQ_ERR_NOMEM : CFPQ_OK;
}

}  // namespace cfpq
