// C ABI of the CFPQ engine: contexts, the fixpoint loop of Algorithm 1 (Section 4.2) as a
// CUDA graph with a conditional while node, and result extraction (R_A, Section 2).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "cfpq_device.cuh"
#include "cfpq_internal.h"
#include "cfpq_lengths.cuh"

namespace cfpq {

// ------------------------------------------------------------------------------------
// Kernels (thin wrappers over the device functions of cfpq_device.cuh)
// ------------------------------------------------------------------------------------

__global__ void k_seed(const QDesc *qd) {
    const QDesc q = *qd;
    seed_query(q, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
}

// Product item of the single-query gather list: group (6 bits), column chunk (5), row (17).
__device__ __forceinline__ uint32_t pack_row_item(int g, uint32_t ch, uint32_t i) {
    return ((uint32_t)g << 22) | (ch << 17) | i;
}

// Gather scan for the loop execution of parity par (one lane per (group, row word)): the rows
// of the word that have a left delta row or, where the right operand has a delta, a non-empty
// left row, become one list item per column chunk. Every group is listed; the gather skips
// the groups that the execution's choice puts on the tensor cores.
__device__ __forceinline__ void scan_rows(const QDesc &q, uint64_t item, uint32_t par, uint32_t *list, uint32_t cap,
                                          uint32_t nch) {
    DevState *st = q.st;
    const uint32_t rw = (q.n + 31u) / 32u;
    const int lane = threadIdx.x & 31;
    uint32_t cand = 0, wq = 0;
    int g = 0;
    if (item < (uint64_t)q.n_groups * rw) {
        g = (int)(item / rw);
        wq = (uint32_t)(item % rw);
        const uint32_t *DR = par ? q.R1 : q.R0;
        // the three loads of a production do not depend on one another, nor on the other
        // productions': issued together, a few productions cost one round trip
#pragma unroll 4
        for (int r = q.gstart[g]; r < q.gstart[g + 1]; r++) {
            const int B = q.rules[r].b, C = q.rules[r].c;
            const uint32_t d = __ldcg(DR + (uint64_t)B * q.W + wq);
            const unsigned long long dc = __ldcg(&st->dcount[par][C]);
            const uint32_t t = __ldcg(q.Trow + (uint64_t)B * q.W + wq);
            cand |= d | (dc != 0ull ? t : 0u);
        }
        cand &= rows_in_word(q.n, wq) & rows_of_block(q, wq);
    }
    const uint32_t cnt = (uint32_t)__popc(cand) * nch;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t wtotal = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && wtotal) base = atomicAdd(&st->list_len[par], wtotal);
    base = __shfl_sync(0xffffffffu, base, 31);
    uint32_t pos = base + incl - cnt;
    if ((uint64_t)pos + cnt > cap) {  // cannot happen: the list holds every (group, row, chunk)
        if (cnt) atomicExch(&st->error, kErrTimeout);
        return;
    }
    while (cand) {
        const uint32_t i = wq * 32u + (uint32_t)(__ffs(cand) - 1);
        cand &= cand - 1;
        for (uint32_t ch = 0; ch < nch; ch++) list[pos++] = pack_row_item(g, ch, i);
    }
}

// The first loop execution's list (after the seed).
__global__ void __launch_bounds__(256) k_scan_rows(const QDesc *qd, uint32_t *list, uint32_t cap, uint32_t nch) {
    const QDesc &q = *qd;
    scan_rows(q, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint32_t)(q.st->iter & 1ull), list, cap, nch);
}

// The listed gathers of one loop execution over the warps of the grid (every thread of every
// block calls it).
template <int CPL>
__device__ __forceinline__ void gather_listed(const QDesc &q, const uint32_t *list, uint32_t cap) {
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t gwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const DevState *st = q.st;
    const uint32_t parity = (uint32_t)(st->iter & 1ull);
    const uint32_t len = min(st->list_len[parity], cap);
    uint64_t tensor_groups = 0;  // this execution's tensor-core groups: their listed items are skipped
    for (int g = 0; g < q.n_groups; g++)
        if (st->use_tensor[g]) tensor_groups |= 1ull << g;
    if (gwarp == 0 && lane == 0)
        for (int g = 0; g < q.n_groups; g++)
            if (!((tensor_groups >> g) & 1ull))
                atomicAdd(&q.st->gather_products, (unsigned long long)(q.gstart[g + 1] - q.gstart[g]));
    // new pairs per non-terminal, gathered per block and added to the counts once per block
    // (the items' counts all go to the same few addresses)
    __shared__ unsigned long long s_new[kMaxNT];
    for (int a = threadIdx.x; a < q.n_nt; a += blockDim.x) s_new[a] = 0ull;
    __syncthreads();
    for (uint64_t w = gwarp; w < len; w += gwarps) {
        const uint32_t e = list[w];
        const int g = (int)(e >> 22);
        if ((tensor_groups >> g) & 1ull) continue;
        gather_row_chunk<CPL>(q, g, e & 0x1FFFFu, (e >> 17) & 31u, lane, parity, s_new);
    }
    __syncthreads();
    for (int a = threadIdx.x; a < q.n_nt; a += blockDim.x) {
        const unsigned long long v = s_new[a];
        if (!v) continue;
        atomicAdd(&q.st->dcount[parity ^ 1u][a], v);
        atomicAdd(&q.st->tcount[a], v);
        atomicAdd(&q.st->new_bits, v);
        q.st->changed = 1u;
        q.st->dirty[a] = 1u;
        q.st->odirty[a] = 1u;
    }
}

template <int CPL>
__global__ void __launch_bounds__(256, CPL >= 8 ? 3 : 4) k_gather_list(const QDesc *qd, const uint32_t *list, uint32_t cap,
                                                                       int honor_skip) {
    const QDesc &q = *qd;
    if (honor_skip && ld_u32(&q.st->skip)) return;  // an unrolled loop body past the loop's end
    gather_listed<CPL>(q, list, cap);
}

// Jacobi schedule: T |= N over the rows N touched (T_{k+1} = T_k u T_k x T_k). Persistent grid,
// one warp per flagged row (the lanes test 32 rows of the warp's share at once; four chunks of
// 32 words in flight); the word summary of T follows, and where lengths are kept (TTsum set)
// T^T and its summary too, their bits set one per lane per round.
__device__ __forceinline__ void merge_new_rows(const QDesc &q) {
    const int lane = threadIdx.x & 31;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t gwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t parity = (uint32_t)(q.st->iter & 1ull);
    const uint32_t *NR = parity ? q.R0 : q.R1;
    const uint32_t W = q.W;
    const bool keep_tt = q.TTsum != nullptr;
    const uint64_t total = (uint64_t)q.n_nt * q.n;
    for (uint64_t base = gwarp; base < total; base += 32ull * gwarps) {
        const uint64_t mine = base + (uint64_t)lane * gwarps;
        const bool flagged = mine < total && test_bit(NR + (mine / q.n) * W, (uint32_t)(mine % q.n));
        unsigned rowmask = __ballot_sync(0xffffffffu, flagged);
        while (rowmask) {
            const int src = __ffs(rowmask) - 1;
            rowmask &= rowmask - 1;
            const uint64_t g = base + (uint64_t)src * gwarps;
            const int a = (int)(g / q.n);
            const uint32_t i = (uint32_t)(g % q.n);
            if (lane == 0) atomicOr(&q.Trow[(uint64_t)a * W + (i >> 5)], 1u << (i & 31));
            const uint32_t *N = (parity ? q.X0 : q.X1) + (uint64_t)a * q.plane + (uint64_t)i * W;
            uint32_t *T = q.T + (uint64_t)a * q.plane + (uint64_t)i * W;
            for (uint32_t w0 = 0; w0 < W; w0 += 128) {
                uint32_t nw[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t w = w0 + 32u * u + lane;
                    nw[u] = w < W ? __ldcg(N + w) : 0u;
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t w = w0 + 32u * u + lane;
                    if (nw[u]) T[w] = __ldcg(T + w) | nw[u];
                    const unsigned sb = __ballot_sync(0xffffffffu, nw[u] != 0u);
                    if (lane == 0 && sb && q.Tsum)
                        atomicOr(&q.Tsum[((uint64_t)a * q.n_pad + i) * q.SW + ((w0 + 32u * u) >> 5)], sb);
                    if (!keep_tt) continue;
                    uint32_t x = nw[u];
                    while (__any_sync(0xffffffffu, x != 0u)) {
                        if (x) {
                            const uint64_t j = (uint64_t)w * 32u + (uint32_t)(__ffs(x) - 1);
                            x &= x - 1;
                            atomicOr(q.TT + (uint64_t)a * q.plane + j * W + (i >> 5), 1u << (i & 31));
                            atomicOr(q.TTsum + ((uint64_t)a * q.n_pad + j) * q.SW + (i >> 10), 1u << ((i >> 5) & 31));
                        }
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_merge(const QDesc *qd, int honor_skip) {
    const QDesc &q = *qd;
    if (honor_skip && ld_u32(&q.st->skip)) return;
    merge_new_rows(q);
}

// Start of a solve (the matrix initialisation's first part): the loop state from the context's
// template with the deadline armed, and every word of the three row bitmaps (T and both
// deltas) zeroed; on a context whose last solve converged (clear_t), the rows of T that its
// row bitmap flags are zeroed first, with their summary words (every other row of T, and both
// delta planes, are zero already). One block per (non-terminal, row word); the k-th flagged
// row of the word goes to warp k % 4, which zeroes it with 16-byte stores (W is a multiple of
// 8, SW of 4); block 0 also writes the state.
__global__ void __launch_bounds__(128) k_reset(const QDesc *qd, const DevState *tmpl, unsigned long long dt_ns,
                                               int clear_t) {
    const QDesc &q = *qd;
    if (blockIdx.x == 0) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(tmpl);
        uint32_t *dst = reinterpret_cast<uint32_t *>(q.st);
        for (uint32_t w = threadIdx.x; w < (uint32_t)(sizeof(DevState) / 4); w += blockDim.x) dst[w] = src[w];
        __syncthreads();
        if (threadIdx.x == 0 && dt_ns) q.st->deadline_ns = globaltimer_ns() + dt_ns;
    }
    const int a = (int)(blockIdx.x / q.W);
    const uint32_t wq = blockIdx.x % q.W;
    const uint64_t word = (uint64_t)a * q.W + wq;
    if (clear_t && wq < (q.n + 31u) / 32u) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        uint32_t rows = __ldcg(q.Trow + word) & rows_in_word(q.n, wq);
        uint4 *T = reinterpret_cast<uint4 *>(q.T + (uint64_t)a * q.plane);
        const uint32_t W4 = q.W / 4u, SW4 = q.SW / 4u;
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        for (int k = 0; rows; k++) {
            const uint64_t i = wq * 32u + (uint32_t)(__ffs(rows) - 1);
            rows &= rows - 1;
            if ((k & 3) != warp) continue;
            for (uint32_t w = (uint32_t)lane; w < W4; w += 32u) T[i * W4 + w] = z;
            if (q.Tsum) {
                uint4 *sum = reinterpret_cast<uint4 *>(q.Tsum + ((uint64_t)a * q.n_pad + i) * q.SW);
                for (uint32_t w = (uint32_t)lane; w < SW4; w += 32u) sum[w] = z;
            }
        }
        __syncthreads();  // every warp has read the word
    }
    if (threadIdx.x == 0) {
        q.Trow[word] = 0u;
        q.R0[word] = 0u;
        q.R1[word] = 0u;
    }
}

// Clears the rows of the delta plane read in this execution. Blocks take (non-terminal, row
// word of 32 rows) units grid-stride (block b of nb); the k-th flagged row of a unit goes to
// warp k % (warps per block), which zeroes it with 16-byte stores (W is a multiple of 8, so
// every row is whole uint4s).
__device__ __forceinline__ void clear_delta_rows(const QDesc &q, uint32_t b, uint32_t nb, uint32_t parity) {
    const uint32_t rw = (q.n + 31u) / 32u;
    const uint32_t W4 = q.W / 4u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    const uint32_t *DR = parity ? q.R1 : q.R0;
    for (uint32_t unit = b; unit < (uint32_t)q.n_nt * rw; unit += nb) {
        const int a = (int)(unit / rw);
        const uint32_t wq = unit % rw;
        uint32_t rows = __ldcg(DR + (uint64_t)a * q.W + wq) & rows_in_word(q.n, wq);
        uint4 *D = reinterpret_cast<uint4 *>((parity ? q.X1 : q.X0) + (uint64_t)a * q.plane);
        for (int k = 0; rows; k++) {
            const uint64_t i = wq * 32u + (uint32_t)(__ffs(rows) - 1);
            rows &= rows - 1;
            if (k % nw != warp) continue;
            for (uint32_t w = (uint32_t)lane; w < W4; w += 32u) D[i * W4 + w] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

// The same clear for one (non-terminal, row word) unit by one warp: it reads the unit's word
// of the read row bitmap, zeroes that word (so the tail need not zero the bitmap), and zeroes
// the flagged rows.
__device__ __forceinline__ void clear_delta_unit_warp(const QDesc &q, uint64_t unit, uint32_t parity) {
    const uint32_t rw = (q.n + 31u) / 32u;
    const uint32_t W4 = q.W / 4u;
    const int lane = threadIdx.x & 31;
    const uint64_t a = unit / rw;
    const uint32_t wq = (uint32_t)(unit % rw);
    uint32_t *word = (parity ? q.R1 : q.R0) + a * q.W + wq;
    const uint32_t v = __ldcg(word);
    __syncwarp();
    if (lane == 0 && v) *word = 0u;
    uint32_t rows = v & rows_in_word(q.n, wq);
    uint4 *D = reinterpret_cast<uint4 *>((parity ? q.X1 : q.X0) + a * q.plane);
    while (rows) {
        const uint64_t i = wq * 32u + (uint32_t)(__ffs(rows) - 1);
        rows &= rows - 1;
        for (uint32_t w = (uint32_t)lane; w < W4; w += 32u) D[i * W4 + w] = make_uint4(0u, 0u, 0u, 0u);
    }
}

__global__ void __launch_bounds__(128) k_clear(const QDesc *qd, int honor_skip) {
    if (honor_skip && ld_u32(&qd->st->skip)) return;
    clear_delta_rows(*qd, blockIdx.x, gridDim.x, (uint32_t)(qd->st->iter & 1ull));
}

// End of a loop execution on a path with gathers: blocks below scan_blocks list the next
// execution's gather items (its delta rows and counts are final here), the others clear the
// delta rows read in this execution (the two touch different planes).
__global__ void __launch_bounds__(256) k_clear_scan(const QDesc *qd, uint32_t *list, uint32_t cap, uint32_t nch,
                                                    uint32_t scan_blocks, int honor_skip) {
    const QDesc &q = *qd;
    if (honor_skip && ld_u32(&q.st->skip)) return;
    if (blockIdx.x < scan_blocks)
        scan_rows(q, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint32_t)((q.st->iter + 1ull) & 1ull), list,
                  cap, nch);
    else
        clear_delta_rows(q, blockIdx.x - scan_blocks, gridDim.x - scan_blocks, (uint32_t)(q.st->iter & 1ull));
}


// AUTO path, start of a loop execution (one thread per group): for every production group, the
// cheaper of the two product kinds by a cost model on the device-side counts, and which group
// refreshes each transpose that a tensor product will read. Gather cost: one right-operand row
// (W words) per bit of D_B, plus, where the right operand has a delta, a scan of the non-empty
// rows of T_B (2W words each) and one D_C row per bit of T_B that meets a non-empty row of D_C
// (expected |T_B| * min(1, |D_C| / n)). Tensor cost, per production: with tile skipping and
// both operands' tile counts known, the live K steps sum_k mB[k] nC[k] (mB[k]: m-tiles of T_B
// whose K slice k is non-zero; nC[k]: n-tiles of T_C^T) at the measured rate of executed work
// with skipping; otherwise the dense 2 n_pad^3 at the dense rate of the operand kind; plus a
// transpose per right operand changed since its last refresh and the launches. When the gather
// has become expensive (kProbeNs) and the dense price is higher still, the counts that tile
// skipping would need are asked for (occ_probe: the next execution's occupancy pass runs even
// if no group takes the tensor cores), so the next choice prices the live steps.
// Measured rates (Boolean ops per ns) of dense products and of the work executed with tile
// skipping, for E4M3 and E2M1 operands.
__device__ __forceinline__ float tensor_ops_per_ns(int kind) { return kind ? 7.6e6f : 3.2e6f; }
__device__ __forceinline__ float skip_ops_per_ns(int kind) { return kind ? 3.2e6f : 2.2e6f; }
constexpr float kStepOps = 2.0f * 128.0f * 256.0f * 128.0f;  // Boolean ops of one K slice of a tile
constexpr float kTensorLaunchNs = 8000.0f;               // plan and product launches of a group
constexpr float kProbeNs = 100000.0f;
constexpr float kGatherBytesPerNs = 600.0f;   // measured gather rate (latency-bound)
constexpr float kTransposeBytesPerNs = 3000.0f;

// Every thread of one block (at least max(n_nt, n_groups) threads) calls this: thread g
// costs group g from the device-side counts, thread a assigns the refresh of TT[A].
// Live K steps of a production with tile skipping: the dot product of its operands' per-slice
// tile counts, one warp per production (the first kLiveRules) and the lanes over the slices.
// The counts are integers and the sums stay below 2^24, so the float sums are exact in any order.
constexpr int kLiveRules = 256;
__device__ __forceinline__ float live_steps_of(const QDesc &q, int B, int C, int lane) {
    const uint32_t *mB = q.occCA + (uint64_t)B * q.KS, *nC = q.occCB + (uint64_t)C * q.KS;
    float live = 0.0f;
    for (uint32_t k = (uint32_t)lane; k < q.KS; k += 32u) live += (float)__ldcg(mB + k) * (float)__ldcg(nC + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) live += __shfl_xor_sync(0xffffffffu, live, o);
    return live;
}

__device__ void choose_products(const QDesc &q, const cudaGraphConditionalHandle *handles, int use_handles) {
    __shared__ unsigned s_use[kMaxNT], s_any, s_probe;
    __shared__ float s_live[kLiveRules];
    // the per-non-terminal counts and flags the costs read, loaded at once (nothing changes
    // them while the choice runs)
    __shared__ float s_dc[kMaxNT], s_tc[kMaxNT];
    __shared__ unsigned s_dirty[kMaxNT], s_known[kMaxNT];
    // the productions' operands (the first kLiveRules) and the group starts, in the same round
    // trip as the counts
    __shared__ int2 s_bc[kLiveRules];
    __shared__ int s_gstart[kMaxNT + 1];
    DevState *st = q.st;
    const int tid = threadIdx.x;
    const unsigned long long it = ld_u64(&st->iter);
    if (tid == 0) s_any = s_probe = 0u;
    if (tid < q.n_nt) {
        // both parities' delta counts, loaded beside the iteration number (not after it)
        const unsigned long long d0 = ld_u64(&st->dcount[0][tid]), d1 = ld_u64(&st->dcount[1][tid]);
        s_tc[tid] = (float)ld_u64(&st->tcount[tid]);
        s_dirty[tid] = ld_u32(&st->dirty[tid]);
        s_known[tid] = q.occKnown ? ld_u32(&q.occKnown[tid]) : 0u;
        s_dc[tid] = (float)((it & 1ull) ? d1 : d0);
    }
    for (int r = tid; r < q.n_rules && r < kLiveRules; r += (int)blockDim.x) s_bc[r] = make_int2(q.rules[r].b, q.rules[r].c);
    for (int g = tid; g <= q.n_groups; g += (int)blockDim.x) s_gstart[g] = q.gstart[g];
    __syncthreads();
    auto operands = [&](int r) { return r < kLiveRules ? s_bc[r] : make_int2(q.rules[r].b, q.rules[r].c); };
    if (q.occA)
        for (int r = tid >> 5; r < q.n_rules && r < kLiveRules; r += (int)(blockDim.x >> 5)) {
            const int B = s_bc[r].x, C = s_bc[r].y;
            const float live = (s_known[B] && s_known[C]) ? live_steps_of(q, B, C, tid & 31) : 0.0f;
            if ((tid & 31) == 0) s_live[r] = live;
        }
    __syncthreads();
    if (tid < q.n_groups) {
        const int g = tid;
        // single precision: a cost estimate (either choice is exact), and FP32 is the fast pipe
        const int kind = q.tensor_kind == CFPQ_TENSOR_FP8 ? 0 : 1;
        const float n = (float)q.n, W = (float)q.W, np = (float)q.n_pad;
        const float dense_rule_ns = 2.0f * np * np * np / tensor_ops_per_ns(kind);
        // a transpose reads T_C (n^2 / 8 bytes) and writes T_C^T: as nibbles (n^2 / 2 bytes)
        // for dense E2M1 products (no tile occupancy), bit-packed otherwise
        const bool nibble = kind && !q.occA;
        const float transpose_ns = (np * np / 8.0f + (nibble ? np * np / 2.0f : np * np / 8.0f)) / kTransposeBytesPerNs;
        const int r0 = s_gstart[g], r1 = s_gstart[g + 1];
        float words = 0.0f, tensor_ns = kTensorLaunchNs;
        bool unknown = false;
        for (int r = r0; r < r1; r++) {
            const int2 bc = operands(r);
            const int B = bc.x, C = bc.y;
            const float dB = s_dc[B], dC = s_dc[C], tB = s_tc[B];
            words += dB * W;
            if (dC > 0.0f) words += fminf(n, tB) * 2.0f * W + tB * fminf(1.0f, dC / n) * W;
            const float extra = s_dirty[C] ? transpose_ns : 0.0f;
            if (q.occA && s_known[B] && s_known[C]) {
                float live = 0.0f;
                if (r < kLiveRules) {
                    live = s_live[r];
                } else {  // beyond the warps' productions: this thread alone
                    const uint32_t *mB = q.occCA + (uint64_t)B * q.KS, *nC = q.occCB + (uint64_t)C * q.KS;
                    for (uint32_t k = 0; k < q.KS; k++) live += (float)__ldcg(mB + k) * (float)__ldcg(nC + k);
                }
                tensor_ns += live * kStepOps / skip_ops_per_ns(kind) + extra;
            } else {
                tensor_ns += dense_rule_ns + extra;
                unknown = true;
            }
        }
        const float gather_ns = words * 4.0f / kGatherBytesPerNs;
        const unsigned use = tensor_ns < gather_ns ? 1u : 0u;
        // an occupancy pass reads each operand's plane once: worth it only where it is small
        // against the gather it may replace
        const float pass_ns = 2.0f * (float)(r1 - r0) * np * np / 8.0f / kTransposeBytesPerNs;
        if (q.occA && unknown && !use && gather_ns > fmaxf(kProbeNs, 10.0f * pass_ns)) {
            // tile skipping might beat the gather here: the next occupancy pass gets these counts
            for (int r = r0; r < r1; r++) {
                const int2 bc = operands(r);
                st->occ_now[bc.x] = st->occ_now[bc.y] = 1u;
            }
            atomicOr(&s_probe, 1u);
        }
        st->use_tensor[g] = use;
        s_use[g] = use;
        if (use_handles) cudaGraphSetConditional(handles[g], use);
        if (use) atomicOr(&s_any, 1u);
    }
    __syncthreads();
    if (tid == 0) {
        st->occ_probe = s_probe;
        st->any_next = s_any | s_probe;
    }
    if (tid == 0 && use_handles) cudaGraphSetConditional(handles[q.n_groups], s_any | s_probe);

    if (tid < q.n_nt) {
        // the first group (in order) taking the tensor product with A as a right operand
        // refreshes TT[A] if A changed since its last refresh
        const int a = tid;
        unsigned owner = 0u;
        for (int g = 0; g < q.n_groups && !owner; g++)
            if (s_use[g])
                for (int r = s_gstart[g]; r < s_gstart[g + 1]; r++)
                    if (operands(r).y == a) {
                        owner = (unsigned)g + 1u;
                        break;
                    }
        const unsigned now = (owner != 0u && s_dirty[a]) ? owner : 0u;
        st->tt_now[a] = now;
        if (now) st->dirty[a] = 0u;
    }
    __syncthreads();
}

// The choice before the loop. nested (the graph's nested loops): the inner loop's handle and
// skip follow the choice, as the tail sets them after every execution.
__global__ void k_choose(const QDesc *qd, const cudaGraphConditionalHandle *handles, int use_handles, int nested) {
    const QDesc &q = *qd;
    choose_products(q, handles, use_handles);
    if (nested && threadIdx.x == 0) {
        const unsigned any = ld_u32(&q.st->any_next);
        cudaGraphSetConditional(handles[q.n_groups + 1], any ? 0u : 1u);
        q.st->skip = any ? 1u : 0u;
    }
}

// End of a loop execution. choice != NULL (automatic path in a graph): the product choice for
// the next execution is made here too, saving a launch per execution.
// flags: kTailHonorSkip, the tail of an unrolled body's copy (nothing to do once skip is set);
// kTailUnrolled, the body repeats the execution and the copies after this one skip once the
// loop ends; kTailNested (AUTO, with choice), the body runs gather-only executions in an inner
// loop on handle choice[n_groups + 1] and a mixed one under the IF on choice[n_groups]: both
// handles and skip follow the next execution's product choice.
enum : int { kTailHonorSkip = 1, kTailUnrolled = 2, kTailNested = 4 };

__global__ void k_tail(const QDesc *qd, cudaGraphConditionalHandle handle, int use_handle,
                       const cudaGraphConditionalHandle *choice, int flags) {
    const QDesc &q = *qd;
    if ((flags & kTailHonorSkip) && ld_u32(&q.st->skip)) return;
    const unsigned cont = tail_query(q, threadIdx.x, blockDim.x, true);
    if (cont && choice) choose_products(q, choice, 1);
    if (threadIdx.x == 0) {
        if (use_handle) cudaGraphSetConditional(handle, cont);
        if (flags & kTailNested) {
            const unsigned any = cont ? ld_u32(&q.st->any_next) : 0u;
            const unsigned gather_only = cont && !any ? 1u : 0u;
            cudaGraphSetConditional(choice[q.n_groups], any);  // no tensor branch after the loop's end
            cudaGraphSetConditional(choice[q.n_groups + 1], gather_only);
            q.st->skip = gather_only ? 0u : 1u;
        } else if (flags & kTailUnrolled) {
            q.st->skip = cont ? 0u : 1u;
        }
    }
}


// Gather-only loop executions in one persistent launch (every block resident: a cooperative
// launch of 256-thread blocks). Each execution runs the work of the launches it replaces in
// phases separated by grid barriers: the listed gathers; (LEN) the lengths of the pairs they
// added, read from T before the merge; (Jacobi) the merge T |= N, which the
// next list reads through the row bitmap of T; then, at once, block 0's tail (the loop
// condition and, with choice, the next execution's product choice) and, on the other blocks'
// warps, the next execution's list and the clear of the delta rows read (each clear unit also
// zeroing its word of the read row bitmap, which the tail zeroes otherwise). The tail reads only what the gathers (and the
// merge) wrote, and writes nothing the clear or the list reads: the counts of the parity just
// read, the iteration number (each block took the parity before the execution), the choice.
// The launch ends when the loop ends or (choice) the next execution has a tensor product; on
// the way out block 0 sets the graph's handles as k_tail does with the same flags
// (kTailNested: the nested loops'; kTailUnrolled: the loop's alone).
template <int CPL, bool LEN>
__global__ void __launch_bounds__(256, CPL >= 8 ? 3 : 4)
    k_gather_loop(const QDesc *qd, uint32_t *list, uint32_t cap, uint32_t nch, cudaGraphConditionalHandle handle,
                  const cudaGraphConditionalHandle *choice, int flags, uint32_t *L, uint32_t *Wit, uint64_t lplane) {
    const QDesc &q = *qd;
    DevState *st = q.st;
    __shared__ unsigned long long s_target;
    __shared__ unsigned s_go;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->loop_launches, 1u);
    grid_sync_start(st, s_target);
    const bool jacobi = q.schedule == CFPQ_SCHED_JACOBI;
    // the clear and the list: warps of blocks 1 .. (block 0 runs the tail), the list's
    // (group, row word) items 32 to a warp, then the clear's (non-terminal, row word) units one
    // to a warp
    const uint32_t rw = (q.n + 31u) / 32u;
    const uint32_t first = gridDim.x > 1 ? 1u : 0u;
    const uint64_t warps = (uint64_t)(gridDim.x - first) * (blockDim.x >> 5);
    const uint64_t my_warp = (uint64_t)(blockIdx.x - first) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t scan_warps = ((uint64_t)q.n_groups * rw + 31u) / 32u;  // 32 items each
    const uint64_t clear_warps = (uint64_t)q.n_nt * rw;                   // one unit each
    for (;;) {
        const uint32_t par = (uint32_t)(ld_u64(&st->iter) & 1ull);  // this execution's parity
        gather_listed<CPL>(q, list, cap);
        if (!grid_sync(st, s_target)) break;
        if constexpr (LEN) {  // the new pairs' lengths, from T before the merge (Section 5)
            lengths_of_new_pairs(q, L, Wit, lplane);
            if (!grid_sync(st, s_target)) break;
        }
        if (jacobi) {
            merge_new_rows(q);
            if (!grid_sync(st, s_target)) break;
        }
        if (blockIdx.x == 0) {
            const unsigned cont = tail_query(q, threadIdx.x, blockDim.x, false);
            // the per-group handles matter only to a mixed execution: set on the way out
            if (cont && choice) choose_products(q, choice, 0);
            if (threadIdx.x == 0) {
                const unsigned any = (cont && choice) ? ld_u32(&st->any_next) : 0u;
                const unsigned go = cont && !any ? 1u : 0u;
                st->loop_execs += 1ull;
                if (!go) {
                    cudaGraphSetConditional(handle, cont);
                    if (any)
                        for (int g = 0; g < q.n_groups; g++) cudaGraphSetConditional(choice[g], st->use_tensor[g]);
                    if (flags & kTailNested) {
                        cudaGraphSetConditional(choice[q.n_groups], any);
                        cudaGraphSetConditional(choice[q.n_groups + 1], 0u);
                    }
                    st->skip = 1u;
                }
                st->loop_go = go;  // read by every block after the barrier
            }
        }
        if (blockIdx.x >= first)
            for (uint64_t w = my_warp; w < scan_warps + clear_warps; w += warps) {
                if (w < scan_warps)
                    scan_rows(q, w * 32u + (threadIdx.x & 31u), par ^ 1u, list, cap, nch);
                else
                    clear_delta_unit_warp(q, w - scan_warps, par);
            }
        if (!grid_sync(st, s_target)) break;
        if (threadIdx.x == 0) s_go = ld_u32(&st->loop_go) && ld_u32(&st->error) != kErrDevice;
        __syncthreads();
        if (!s_go) break;
    }
    // a barrier that gave up (kErrDevice): the loop stops here, so that no conditional node
    // runs this launch again
    if (blockIdx.x == 0 && threadIdx.x == 0 && ld_u32(&st->error) == kErrDevice) {
        cudaGraphSetConditional(handle, 0u);
        if (flags & kTailNested) {
            cudaGraphSetConditional(choice[q.n_groups], 0u);
            cudaGraphSetConditional(choice[q.n_groups + 1], 0u);
        }
        st->skip = 1u;
        st->cont = 0u;
        st->done = 1u;
    }
}

__global__ void k_arm_deadline(DevState *st, unsigned long long dt_ns) { st->deadline_ns = globaltimer_ns() + dt_ns; }

// --- sharded solve by row blocks: the exchange of one loop execution's new pairs ---

// Records of the pairs that this execution's products added to the context's rows: a record is
// [A, i, the W words of row i of N_A]. One warp per (non-terminal, row word of 32 rows) of the
// block; the word of the new delta's row bitmap flags the rows to pack. Records beyond
// cap_records are counted but not written.
__global__ void __launch_bounds__(256) k_block_pack(const QDesc *qd, uint32_t *out, uint64_t cap_records) {
    const QDesc &q = *qd;
    DevState *st = q.st;
    const uint32_t parity = (uint32_t)(st->iter & 1ull);
    const uint32_t *NR = parity ? q.R0 : q.R1;
    const uint32_t *N = parity ? q.X0 : q.X1;
    const uint32_t W = q.W, rec_words = 2u + W;
    const int lane = threadIdx.x & 31;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t gwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t w0 = q.row0 / 32u, nw = (min(q.row1, q.n) + 31u) / 32u - w0;  // row words of the block
    for (uint64_t u = gwarp; u < (uint64_t)q.n_nt * nw; u += gwarps) {
        const int a = (int)(u / nw);
        const uint32_t wq = w0 + (uint32_t)(u % nw);
        uint32_t rows = __ldcg(NR + (uint64_t)a * W + wq) & rows_in_word(q.n, wq);
        while (rows) {
            const uint32_t i = wq * 32u + (uint32_t)(__ffs(rows) - 1);
            rows &= rows - 1;
            unsigned long long slot = 0;
            if (lane == 0) slot = atomicAdd(&st->block_records, 1ull);
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (slot >= cap_records) continue;
            uint32_t *rec = out + slot * rec_words;
            if (lane == 0) {
                rec[0] = (uint32_t)a;
                rec[1] = i;
            }
            const uint32_t *row = N + (uint64_t)a * q.plane + (uint64_t)i * W;
            for (uint32_t w = lane; w < W; w += 32u) rec[2 + w] = __ldcg(row + w);
        }
    }
}

// Another rank's records ORed into this execution's new pairs, as a product epilogue adds
// them (delta plane, its row bitmap, the counts and change flags), so that the merge and the
// next execution treat them like the context's own. One warp per record.
__global__ void __launch_bounds__(256) k_block_import(const QDesc *qd, const uint32_t *in, uint64_t n_records) {
    const QDesc &q = *qd;
    DevState *st = q.st;
    const uint32_t parity = (uint32_t)(st->iter & 1ull);
    uint32_t *NR = parity ? q.R0 : q.R1;
    uint32_t *N = parity ? q.X0 : q.X1;
    const uint32_t W = q.W, rec_words = 2u + W;
    const int lane = threadIdx.x & 31;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t gwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r = gwarp; r < n_records; r += gwarps) {
        const uint32_t *rec = in + r * rec_words;
        const uint32_t a = __ldcg(rec), i = __ldcg(rec + 1);
        if (a >= (uint32_t)q.n_nt || i >= q.n) {
            if (lane == 0) st->block_bad = 1u;
            continue;
        }
        uint32_t *row = N + (uint64_t)a * q.plane + (uint64_t)i * W;
        unsigned cnt = 0;
        for (uint32_t w = lane; w < W; w += 32u) {
            const uint32_t x = __ldcg(rec + 2 + w);
            if (!x) continue;
            const uint32_t old = __ldcg(row + w);
            const uint32_t nwv = x & ~old;
            if (nwv) {
                row[w] = old | nwv;
                cnt += __popc(nwv);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0 && cnt) {
            atomicOr(&NR[(uint64_t)a * W + (i >> 5)], 1u << (i & 31));
            atomicAdd(&st->dcount[parity ^ 1u][a], (unsigned long long)cnt);
            atomicAdd(&st->tcount[a], (unsigned long long)cnt);
            atomicAdd(&st->new_bits, (unsigned long long)cnt);
            st->changed = 1u;
            st->dirty[a] = 1u;
            st->odirty[a] = 1u;
        }
    }
}

// --- extraction: popc per row -> exclusive scan -> emit (A, m, n) in row-major order ---

// Emits the pairs of row i of T_a (W words) as triples (a, i, j) from position off on, in
// column order (one warp). Eight 32-word chunks are loaded at once, then each non-empty chunk
// is placed by a warp prefix sum of its words' bit counts; empty chunks cost no scan.
__device__ __forceinline__ void emit_row(const uint32_t *row, uint32_t W, int a, uint32_t i, uint64_t off, int lane,
                                         cfpq_triple *out) {
    constexpr int kBatch = 8;
    for (uint32_t b0 = 0; b0 < W; b0 += 32u * kBatch) {
        uint32_t xs[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; k++) {
            const uint32_t w = b0 + 32u * k + (uint32_t)lane;
            xs[k] = w < W ? row[w] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kBatch; k++) {
            uint32_t x = xs[k];
            if (__ballot_sync(0xffffffffu, x != 0u) == 0u) continue;  // warp-uniform
            const uint32_t w0 = b0 + 32u * k;
            const uint32_t c = __popc(x);
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            uint64_t pos = off + incl - c;
            while (x) {
                const uint32_t j = (w0 + lane) * 32u + (uint32_t)(__ffs(x) - 1);
                x &= x - 1;
                out[pos++] = cfpq_triple{a, i, j};
            }
            off += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

__global__ void k_count_rows(const QDesc *qd, int a, uint32_t *counts) {
    const QDesc &q = *qd;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= q.n_pad) return;
    const uint32_t *row = q.T + (uint64_t)a * q.plane + warp * q.W;
    uint32_t c = 0;
    if (test_bit(q.Trow + (uint64_t)a * q.W, (uint32_t)warp))
        for (uint32_t w = lane; w < q.W; w += 32) c += __popc(row[w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) counts[warp] = c;
}

// one block of 1024 threads
// Inclusive prefix sum of one value per thread over a block of 1024 threads: a shuffle scan
// in each warp, then one over the 32 warp totals (ws: 32 shared words), two barriers in all.
__device__ __forceinline__ unsigned long long block_inclusive_scan(unsigned long long x, unsigned long long *ws) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    return x + (w > 0 ? ws[w - 1] : 0ull);
}

__global__ void __launch_bounds__(1024) k_scan(const uint32_t *counts, uint64_t *offsets, uint32_t n,
                                               unsigned long long *total) {
    __shared__ unsigned long long ws[32];
    const uint32_t per = (n + 1023) / 1024;
    const uint32_t lo = threadIdx.x * per, hi = min(n, lo + per);
    unsigned long long s = 0;
    for (uint32_t i = lo; i < hi; i++) s += counts[i];
    const unsigned long long incl = block_inclusive_scan(s, ws);
    unsigned long long run = incl - s;  // exclusive prefix of this segment
    for (uint32_t i = lo; i < hi; i++) {
        offsets[i] = run;
        run += counts[i];
    }
    if (threadIdx.x == 1023) *total = incl;
}

__global__ void k_emit(const QDesc *qd, int a, const uint64_t *offsets, const uint32_t *counts,
                       cfpq_triple *out) {
    const QDesc &q = *qd;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= q.n_pad || counts[warp] == 0) return;
    const uint32_t *row = q.T + (uint64_t)a * q.plane + warp * q.W;
    emit_row(row, q.W, a, (uint32_t)warp, offsets[warp], lane, out);
}

// --- extraction of every relation at once: counts over (non-terminal, row) cells, a
// device-wide three-pass scan, then emission sorted by (A, m, n) ---

__global__ void k_count_all(const QDesc *qd, uint32_t *counts) {
    const QDesc &q = *qd;
    const uint64_t cell = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= (uint64_t)q.n_nt * q.n_pad) return;
    const uint32_t a = (uint32_t)(cell / q.n_pad), i = (uint32_t)(cell % q.n_pad);
    uint32_t c = 0;
    if (i < q.n && test_bit(q.Trow + (uint64_t)a * q.W, i)) {
        const uint32_t *row = q.T + (uint64_t)a * q.plane + (uint64_t)i * q.W;
        for (uint32_t w = lane; w < q.W; w += 32) c += __popc(row[w]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) counts[cell] = c;
}

// pass 1: per-block sums of kScanSeg cells
__global__ void __launch_bounds__(1024) k_scan_blocks(const uint32_t *counts, uint64_t n, unsigned long long *bsum) {
    __shared__ unsigned long long red[32];
    const uint64_t lo = (uint64_t)blockIdx.x * kScanSeg;
    unsigned long long s = 0;
    for (uint64_t i = lo + threadIdx.x; i < min(n, lo + kScanSeg); i += blockDim.x) s += counts[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = red[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = s;
    }
}

// pass 2 (one block): exclusive scan of the block sums; bsum[nb] = total
__global__ void __launch_bounds__(1024) k_scan_bsums(unsigned long long *bsum, int nb, unsigned long long *total) {
    __shared__ unsigned long long ws[32];
    const int t = threadIdx.x;
    const unsigned long long mine = t < nb ? bsum[t] : 0ull;
    const unsigned long long incl = block_inclusive_scan(mine, ws);
    if (t < nb) bsum[t] = incl - mine;
    if (t == 1023) {
        bsum[nb] = incl;
        *total = incl;
    }
}

// pass 3: offsets inside each block's segment (each thread a contiguous run of 8 cells)
__global__ void __launch_bounds__(1024) k_scan_apply(const uint32_t *counts, uint64_t n, const unsigned long long *bsum,
                                                     uint64_t *offsets) {
    __shared__ unsigned long long ws[32];
    const int t = threadIdx.x;
    const uint64_t lo = (uint64_t)blockIdx.x * kScanSeg + (uint64_t)t * (kScanSeg / 1024);
    unsigned long long s = 0;
    for (uint64_t i = lo; i < min(n, lo + kScanSeg / 1024); i++) s += counts[i];
    const unsigned long long incl = block_inclusive_scan(s, ws);
    unsigned long long run = bsum[blockIdx.x] + incl - s;
    for (uint64_t i = lo; i < min(n, lo + kScanSeg / 1024); i++) {
        offsets[i] = run;
        run += counts[i];
    }
}

// first triple of each non-terminal; nt_off[n_nt] = total
__global__ void k_nt_offsets(const QDesc *qd, const uint64_t *offsets, const unsigned long long *total,
                             unsigned long long *nt_off) {
    const QDesc &q = *qd;
    const int a = threadIdx.x;
    if (a < q.n_nt) nt_off[a] = offsets[(uint64_t)a * q.n_pad];
    if (a == q.n_nt) nt_off[a] = *total;
}

__global__ void k_emit_all(const QDesc *qd, const uint64_t *offsets, const uint32_t *counts, cfpq_triple *out) {
    const QDesc &q = *qd;
    const uint64_t cell = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= (uint64_t)q.n_nt * q.n_pad || counts[cell] == 0) return;
    const int a = (int)(cell / q.n_pad);
    const uint32_t i = (uint32_t)(cell % q.n_pad);
    const uint32_t *row = q.T + (uint64_t)a * q.plane + (uint64_t)i * q.W;
    emit_row(row, q.W, a, i, offsets[cell], lane, out);
}

}  // namespace cfpq

using namespace cfpq;

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------

static void note_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    if (getenv("CFPQ_VERBOSE")) fprintf(stderr, "cfpq: %s failed: %s (%s:%d)\n", what, cudaGetErrorString(e), file, line);
}

#define CK(call)                                               \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) {                               \
            note_cuda_error(e_, #call, __FILE__, __LINE__);    \
            return CFPQ_ERR_CUDA;                              \
        }                                                      \
    } while (0)

extern "C" const char *cfpq_strerror(int code) {
    switch (code) {
        case CFPQ_OK: return "ok";
        case CFPQ_ERR_INVALID: return "invalid argument";
        case CFPQ_ERR_NOMEM: return "out of memory";
        case CFPQ_ERR_NOT_SOLVED: return "not solved";
        case CFPQ_ERR_ITER_LIMIT: return "iteration limit reached";
        case CFPQ_ERR_TIMEOUT: return "timeout";
        case CFPQ_ERR_CUDA: return "CUDA error";
        case CFPQ_ERR_BUFFER: return "buffer too small";
        case CFPQ_ERR_UNSUPPORTED: return "unsupported";
        case CFPQ_ERR_NOT_FOUND: return "not found";
        default: return "unknown status";
    }
}

extern "C" int cfpq_options_default(cfpq_options *opt) {
    if (!opt) return CFPQ_ERR_INVALID;
    memset(opt, 0, sizeof(*opt));
    opt->schedule = CFPQ_SCHED_INPLACE;
    opt->path = CFPQ_PATH_AUTO;
    opt->use_graph = 1;
    opt->profile = 0;
    opt->max_iter = 0;
    opt->timeout_s = 0.0;
    return CFPQ_OK;
}

namespace cfpq {

uint32_t gather_chunks(uint32_t W, int *cpl) {
    if (W <= 32) { *cpl = 1; return 1; }
    if (W <= 64) { *cpl = 2; return 1; }
    if (W <= 128) { *cpl = 4; return 1; }
    *cpl = 8;
    return (W + 255) / 256;
}

static uint32_t row_warp_blocks(uint64_t rows) { return (uint32_t)((rows * 32 + 255) / 256); }

// The gather products of one loop execution, for every group not on the tensor cores: a
// persistent grid runs one warp per (group, row, column chunk) item that the list of this
// execution holds (listed after the seed, then at the end of each execution for the next).
static int enqueue_gathers(cfpq_ctx *c, cudaStream_t s, int honor_skip = 0) {
    int cpl;
    gather_chunks(c->W, &cpl);
    const uint32_t grid = (uint32_t)c->gather_grid;
    switch (cpl) {
        case 1: k_gather_list<1><<<grid, 256, 0, s>>>(c->d_q, c->d_list, c->list_cap, honor_skip); break;
        case 2: k_gather_list<2><<<grid, 256, 0, s>>>(c->d_q, c->d_list, c->list_cap, honor_skip); break;
        case 4: k_gather_list<4><<<grid, 256, 0, s>>>(c->d_q, c->d_list, c->list_cap, honor_skip); break;
        default: k_gather_list<8><<<grid, 256, 0, s>>>(c->d_q, c->d_list, c->list_cap, honor_skip); break;
    }
    c->iter_launches += 1;
    CK(cudaGetLastError());
    return CFPQ_OK;
}

// Adds an IF node on handle h to the graph that stream s is capturing (after the capture's
// current dependencies), makes it the capture's only dependency and returns its body.
static int add_cond(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                    cudaGraph_t *body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive) return CFPQ_ERR_CUDA;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, cg, deps, nullptr, nd, &p));
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    *body = p.conditional.phGraph_out[0];
    return CFPQ_OK;
}

static int add_if(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t *body) {
    return add_cond(s, h, cudaGraphCondTypeIf, body);
}

static int begin_branch(cudaStream_t b, cudaGraph_t body) {
    CK(cudaStreamBeginCaptureToGraph(b, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    return CFPQ_OK;
}
static int end_branch(cudaStream_t b, int rc) {
    cudaGraph_t unused = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b, &unused);
    if (rc != CFPQ_OK) return rc;
    CK(e);
    return CFPQ_OK;
}

// AUTO path inside a graph capture on s: the tensor products this execution chose. One IF
// node on "some group chose the tensor product" (on sparse inputs the only node this adds
// per execution) holding one IF node per group: its transposes and tensor product.
static int enqueue_auto_tensor_graph(cfpq_ctx *c, cudaStream_t s) {
    cudaGraph_t any_body;
    int rc = add_if(s, c->h_choice[c->n_groups], &any_body);
    if (rc != CFPQ_OK) return rc;
    if ((rc = begin_branch(c->aux_stream, any_body)) != CFPQ_OK) return rc;
    rc = enqueue_tensor_occupancy(c, c->aux_stream);
    for (int g = 0; g < c->n_groups && rc == CFPQ_OK; g++) {
        cudaGraph_t body;
        if ((rc = add_if(c->aux_stream, c->h_choice[g], &body)) != CFPQ_OK) break;
        if ((rc = begin_branch(c->aux2_stream, body)) != CFPQ_OK) break;
        int r2 = enqueue_tensor_transposes_gated(c, g, c->aux2_stream);
        if (r2 == CFPQ_OK) r2 = enqueue_tensor_group(c, g, c->aux2_stream);
        rc = end_branch(c->aux2_stream, r2);
    }
    return end_branch(c->aux_stream, rc);
}

// One loop execution (the body of Algorithm 1's while loop): the products, then the merge and
// the end of the execution. In profile mode, CUDA events bracket every tensor-product launch
// (one pair per group) and the gather products of the execution (one pair).
static int enqueue_products(cfpq_ctx *c, cudaStream_t s, int use_handle);
static int enqueue_iteration_end(cfpq_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h, int use_handle,
                                 int tail_flags = 0);

int enqueue_iteration(cfpq_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h, int use_handle) {
    c->iter_launches = 0;
    const int rc = enqueue_products(c, s, use_handle);
    if (rc != CFPQ_OK) return rc;
    return enqueue_iteration_end(c, s, h, use_handle);
}

static int enqueue_products(cfpq_ctx *c, cudaStream_t s, int use_handle) {
    const bool prof = c->profile && !use_handle;
    if (c->auto_mixed) {
        // choose per group; in a graph the chosen tensor products run under conditional
        // nodes, otherwise every tensor launch is made and returns at once if not chosen
        if (!use_handle) {  // in the graph, the previous execution's tail (or the node before the loop) chose
            k_choose<<<1, 64, 0, s>>>(c->d_q, nullptr, 0, 0);
            c->iter_launches++;
        }
        if (use_handle) {
            const int rc = enqueue_auto_tensor_graph(c, s);
            if (rc != CFPQ_OK) return rc;
        } else {
            const int orc = enqueue_tensor_occupancy(c, s);
            if (orc != CFPQ_OK) return orc;
            for (int g = 0; g < c->n_groups; g++) {
                int rc = enqueue_tensor_transposes_gated(c, g, s);
                if (rc == CFPQ_OK && prof) rc = enqueue_useful_work(c, g, s);
                if (prof) CK(cudaEventRecord(c->prof_ev[2 * g], s));
                if (rc == CFPQ_OK) rc = enqueue_tensor_group(c, g, s);
                if (prof) CK(cudaEventRecord(c->prof_ev[2 * g + 1], s));
                if (rc != CFPQ_OK) return rc;
            }
        }
    } else {
        if (c->path == CFPQ_PATH_TENSOR) {
            const int orc = enqueue_tensor_occupancy(c, s);
            if (orc != CFPQ_OK) return orc;
        }
        for (int g = 0; g < c->n_groups; g++) {
            if (!c->group_tensor[g]) continue;
            int rc = enqueue_tensor_transposes(c, g, s);
            if (rc == CFPQ_OK && prof) rc = enqueue_useful_work(c, g, s);
            if (prof) CK(cudaEventRecord(c->prof_ev[2 * g], s));
            if (rc == CFPQ_OK) rc = enqueue_tensor_group(c, g, s);
            if (prof) CK(cudaEventRecord(c->prof_ev[2 * g + 1], s));
            if (rc != CFPQ_OK) return rc;
        }
    }
    if (c->any_gather) {
        if (prof) CK(cudaEventRecord(c->prof_ev[2 * c->n_groups], s));
        const int rc = enqueue_gathers(c, s);
        if (prof) CK(cudaEventRecord(c->prof_ev[2 * c->n_groups + 1], s));
        if (rc != CFPQ_OK) return rc;
    }
    return CFPQ_OK;
}

static int enqueue_iteration_end(cfpq_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h, int use_handle,
                                 int tail_flags) {
    const bool prof = c->profile && !use_handle;
    const int honor = (tail_flags & kTailHonorSkip) ? 1 : 0;
    const uint32_t word_blocks = (uint32_t)((uint64_t)c->n_nt * ((c->n + 31) / 32));  // one per (A, row word)
    if (c->lengths) {  // before the merge: T still holds the previous execution's matrices
        if (prof) CK(cudaEventRecord(c->prof_ev[2 * c->n_groups + 2], s));
        const int rc = lengths_enqueue_iteration(c, s);
        if (prof) CK(cudaEventRecord(c->prof_ev[2 * c->n_groups + 3], s));
        if (rc != CFPQ_OK) return rc;
    }
    if (c->schedule == CFPQ_SCHED_JACOBI) {
        const uint64_t blocks_needed = ((uint64_t)c->n_nt * c->n + 7) / 8;  // 8 warps per block
        k_merge<<<(uint32_t)std::min<uint64_t>(blocks_needed, 4ull * (uint64_t)c->sms), 256, 0, s>>>(c->d_q, honor);
        c->iter_launches++;
    }
    if (c->any_gather) {
        int cpl;
        const uint32_t nch = gather_chunks(c->W, &cpl);
        const uint32_t scan_blocks = (uint32_t)(((uint64_t)c->n_groups * ((c->n + 31) / 32) + 255) / 256);
        const uint32_t clear_blocks = std::min<uint32_t>(word_blocks, 2u * (uint32_t)c->sms);
        k_clear_scan<<<scan_blocks + clear_blocks, 256, 0, s>>>(c->d_q, c->d_list, c->list_cap, nch, scan_blocks,
                                                               honor);
    } else {
        k_clear<<<std::min<uint32_t>(word_blocks, 4u * (uint32_t)c->sms), 128, 0, s>>>(c->d_q, honor);
    }
    k_tail<<<1, 1024, 0, s>>>(c->d_q, h, use_handle, (use_handle && c->auto_mixed) ? c->d_choice : nullptr,
                              tail_flags);
    c->iter_launches += 2;
    CK(cudaGetLastError());
    return CFPQ_OK;
}

// profile mode: adds the product launches of the iteration just synchronised. Tensor
// launches count only where the group ran on the tensor cores (AUTO: this execution's choice).
static int collect_profile(cfpq_ctx *c) {
    unsigned used[kMaxNT] = {0};
    if (c->auto_mixed)
        CK(cudaMemcpy(used, c->d_state->use_tensor, sizeof(unsigned) * c->n_groups, cudaMemcpyDeviceToHost));
    for (int g = 0; g < c->n_groups; g++) {
        const bool tensor = c->auto_mixed ? used[g] != 0 : c->group_tensor[g] != 0;
        if (!tensor) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->prof_ev[2 * g], c->prof_ev[2 * g + 1]));
        c->stats.product_ms += ms;
        c->stats.product_launches++;
        c->stats.tensor_ms += ms;
        c->stats.tensor_launches++;
    }
    if (c->any_gather) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->prof_ev[2 * c->n_groups], c->prof_ev[2 * c->n_groups + 1]));
        c->stats.product_ms += ms;
        c->stats.product_launches++;
    }
    if (c->lengths) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->prof_ev[2 * c->n_groups + 2], c->prof_ev[2 * c->n_groups + 3]));
        c->stats.lengths_ms += ms;
        c->stats.lengths_launches++;
    }
    return CFPQ_OK;
}

// Executions per iteration of a graph loop whose executions are gather-only: the copies after
// the one that ends the loop (or, on the automatic path, hands over to a tensor execution)
// return at once, so the loop's count is unchanged and a while-node iteration is paid once per
// kUnroll executions. The first copy always runs (the loop's condition admitted it), so every
// iteration of the loop runs one tail, which sets the condition.
constexpr int kUnroll = 4;

// kUnroll copies of a gather-only execution captured on s (c->iter_launches counts one).
static int capture_gather_executions(cfpq_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h, int tail_flags) {
    int64_t one = 0;
    for (int u = 0; u < kUnroll; u++) {
        c->iter_launches = 0;
        const int honor = u > 0 ? 1 : 0;
        int rc = enqueue_gathers(c, s, honor);
        if (rc == CFPQ_OK) rc = enqueue_iteration_end(c, s, h, 1, tail_flags | (honor ? kTailHonorSkip : 0));
        if (rc != CFPQ_OK) return rc;
        if (u == 0) one = c->iter_launches;
    }
    c->iter_launches = one;
    return CFPQ_OK;
}

// AUTO path, nested loops: one execution in which some group takes the tensor product (or the
// occupancy counts are asked for), captured on s: occupancy, then per group an IF node on its
// choice holding its transposes and tensor product (captured on aux2_stream), the gathers of
// the other groups and the end of the execution.
// The gather-only executions as one persistent launch of k_gather_loop (a cooperative kernel
// node), which runs them until the loop ends or the next one takes a tensor product.
static int capture_gather_loop(cfpq_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h, int tail_flags) {
    int cpl;
    const uint32_t nch = gather_chunks(c->W, &cpl);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.gridDim = dim3((uint32_t)c->loop_grid);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    const QDesc *qd = c->d_q;
    uint32_t *list = c->d_list;
    const uint32_t cap = c->list_cap;
    const cudaGraphConditionalHandle *choice = c->auto_mixed ? c->d_choice : nullptr;
    uint32_t *L = c->d_L, *Wit = c->d_Wit;
    const uint64_t lplane = c->lplane;
    cudaError_t e;
    if (c->lengths) {
        switch (cpl) {
            case 1: e = cudaLaunchKernelEx(&cfg, k_gather_loop<1, true>, qd, list, cap, nch, h, choice, tail_flags, L, Wit, lplane); break;
            case 2: e = cudaLaunchKernelEx(&cfg, k_gather_loop<2, true>, qd, list, cap, nch, h, choice, tail_flags, L, Wit, lplane); break;
            case 4: e = cudaLaunchKernelEx(&cfg, k_gather_loop<4, true>, qd, list, cap, nch, h, choice, tail_flags, L, Wit, lplane); break;
            default: e = cudaLaunchKernelEx(&cfg, k_gather_loop<8, true>, qd, list, cap, nch, h, choice, tail_flags, L, Wit, lplane); break;
        }
    } else {
        switch (cpl) {
            case 1: e = cudaLaunchKernelEx(&cfg, k_gather_loop<1, false>, qd, list, cap, nch, h, choice, tail_flags, L, Wit, lplane); break;
            case 2: e = cudaLaunchKernelEx(&cfg, k_gather_loop<2, false>, qd, list, cap, nch, h, choice, tail_flags, L, Wit, lplane); break;
            case 4: e = cudaLaunchKernelEx(&cfg, k_gather_loop<4, false>, qd, list, cap, nch, h, choice, tail_flags, L, Wit, lplane); break;
            default: e = cudaLaunchKernelEx(&cfg, k_gather_loop<8, false>, qd, list, cap, nch, h, choice, tail_flags, L, Wit, lplane); break;
        }
    }
    if (e != cudaSuccess) {
        note_cuda_error(e, "gather loop", __FILE__, __LINE__);
        return CFPQ_ERR_CUDA;
    }
    return CFPQ_OK;
}

static int capture_mixed_execution(cfpq_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h) {
    int rc = enqueue_tensor_occupancy(c, s);
    for (int g = 0; g < c->n_groups && rc == CFPQ_OK; g++) {
        cudaGraph_t body;
        if ((rc = add_if(s, c->h_choice[g], &body)) != CFPQ_OK) break;
        if ((rc = begin_branch(c->aux2_stream, body)) != CFPQ_OK) break;
        int r2 = enqueue_tensor_transposes_gated(c, g, c->aux2_stream);
        if (r2 == CFPQ_OK) r2 = enqueue_tensor_group(c, g, c->aux2_stream);
        rc = end_branch(c->aux2_stream, r2);
    }
    if (rc == CFPQ_OK && c->any_gather) rc = enqueue_gathers(c, s, 0);
    if (rc == CFPQ_OK) rc = enqueue_iteration_end(c, s, h, 1, kTailNested);
    return rc;
}

// The loop of Algorithm 1 as one graph: a WHILE node on "the last execution changed T" whose
// body is one of
//   automatic path: WHILE (the next execution is gather-only) { kUnroll gather-only
//                   executions, or the persistent loop launch }, then IF (the next one has
//                   a tensor product) { that execution }, after a first choice node;
//   gather-only contexts: kUnroll executions (or the persistent loop launch);
//   otherwise (tensor products every execution; lengths without the persistent loop):
//   one execution.
static int build_graph(cfpq_ctx *c) {
    if (c->graph_exec) return CFPQ_OK;
    bool any_tensor = false;
    for (int g = 0; g < c->n_groups; g++) any_tensor |= c->group_tensor[g] != 0;
    // gather-only executions in one persistent launch where the device can hold its grid;
    // the launch count then comes from the device (loop_launches, loop_execs). Not for a
    // server's contexts: a large query's loop runs beside the grouped launches of the small
    // ones, and a persistent launch would hold every SM until that query converged, where the
    // separate launches interleave with them. Lengths need it for the nested and unrolled
    // shapes (their unrolled copies would run the length kernel past the loop's end).
    const bool persistent = c->loop_grid > 0 && !c->block && !c->pooled;
    const bool nested = c->auto_mixed && (!c->lengths || persistent);
    const bool unrolled = !c->auto_mixed && !any_tensor && c->any_gather && (!c->lengths || persistent);
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(g); note_cuda_error(e, "handle", __FILE__, __LINE__); return CFPQ_ERR_CUDA; }
    cudaGraphNode_t first = nullptr;  // automatic path: the first execution's product choice
    if (c->auto_mixed) {
        // one IF handle per production group, then "any group chose tensor" and (nested) the
        // inner loop's "gather-only", set by the choice before the loop and by every
        // execution's tail for the next one
        const int prc = tensor_prepare(c);
        if (prc != CFPQ_OK) { cudaGraphDestroy(g); return prc; }
        for (cudaStream_t *as : {&c->aux_stream, &c->aux2_stream})
            if (!*as && (e = cudaStreamCreateWithFlags(as, cudaStreamNonBlocking)) != cudaSuccess) {
                cudaGraphDestroy(g);
                note_cuda_error(e, "aux stream", __FILE__, __LINE__);
                return CFPQ_ERR_CUDA;
            }
        // (a handle that no conditional node uses makes the instantiation fail)
        const int handles = c->n_groups + (nested ? 2 : 1);
        c->h_choice.assign(c->n_groups + 2, 0);
        for (int k = 0; k < handles; k++) {
            e = cudaGraphConditionalHandleCreate(&c->h_choice[k], g, 0, 0);
            if (e != cudaSuccess) { cudaGraphDestroy(g); note_cuda_error(e, "choice handle", __FILE__, __LINE__); return CFPQ_ERR_CUDA; }
        }
        e = cudaMemcpy(c->d_choice, c->h_choice.data(), sizeof(cudaGraphConditionalHandle) * (c->n_groups + 2),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaGraphDestroy(g); note_cuda_error(e, "choice copy", __FILE__, __LINE__); return CFPQ_ERR_CUDA; }
        const QDesc *qd = c->d_q;
        const cudaGraphConditionalHandle *hs = c->d_choice;
        int use = 1, nest = nested ? 1 : 0;
        void *args[] = {(void *)&qd, (void *)&hs, (void *)&use, (void *)&nest};
        cudaKernelNodeParams kp = {};
        kp.func = (void *)k_choose;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(64);
        kp.kernelParams = args;
        e = cudaGraphAddKernelNode(&first, g, nullptr, 0, &kp);
        if (e != cudaSuccess) { cudaGraphDestroy(g); note_cuda_error(e, "choice node", __FILE__, __LINE__); return CFPQ_ERR_CUDA; }
    }
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, first ? &first : nullptr, nullptr, first ? 1 : 0, &p);
    if (e != cudaSuccess) { cudaGraphDestroy(g); note_cuda_error(e, "addnode", __FILE__, __LINE__); return CFPQ_ERR_CUDA; }
    cudaGraph_t body = p.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaGraphDestroy(g); note_cuda_error(e, "capture", __FILE__, __LINE__); return CFPQ_ERR_CUDA; }
    int rc = CFPQ_OK;
    if (nested) {
        cudaGraph_t inner = nullptr, mixed = nullptr;
        rc = add_cond(c->stream, c->h_choice[c->n_groups + 1], cudaGraphCondTypeWhile, &inner);
        if (rc == CFPQ_OK && (rc = begin_branch(c->aux_stream, inner)) == CFPQ_OK)
            rc = end_branch(c->aux_stream, persistent ? capture_gather_loop(c, c->aux_stream, h, kTailNested)
                                                      : capture_gather_executions(c, c->aux_stream, h, kTailNested));
        const int64_t per_execution = c->iter_launches;  // a gather-only execution's launches
        if (persistent) c->iter_launches = 0;             // the mixed execution's launches, counted next
        if (rc == CFPQ_OK) rc = add_if(c->stream, c->h_choice[c->n_groups], &mixed);
        if (rc == CFPQ_OK && (rc = begin_branch(c->aux_stream, mixed)) == CFPQ_OK)
            rc = end_branch(c->aux_stream, capture_mixed_execution(c, c->aux_stream, h));
        if (!persistent) c->iter_launches = per_execution;  // else the mixed execution's launches
    } else if (unrolled) {
        if (persistent) {
            rc = capture_gather_loop(c, c->stream, h, kTailUnrolled);
            c->iter_launches = 0;  // every execution runs in the persistent launch
        } else {
            rc = capture_gather_executions(c, c->stream, h, kTailUnrolled);
        }
    } else {
        rc = enqueue_iteration(c, c->stream, h, 1);
    }
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(c->stream, &captured);
    if (rc != CFPQ_OK || e != cudaSuccess) {
        cudaGraphDestroy(g);
        if (e != cudaSuccess) note_cuda_error(e, "endcapture", __FILE__, __LINE__);
        return rc != CFPQ_OK ? rc : CFPQ_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { c->graph_exec = nullptr; note_cuda_error(e, "instantiate", __FILE__, __LINE__); return CFPQ_ERR_CUDA; }
    return CFPQ_OK;
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};
}  // namespace

cudaMemPool_t library_pool(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (g_pool[dev]) return g_pool[dev];
    int supported = 0;
    if (cudaDeviceGetAttribute(&supported, cudaDevAttrMemoryPoolsSupported, dev) != cudaSuccess || !supported) {
        cudaGetLastError();
        return nullptr;
    }
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    // freed memory stays in the pool across synchronisations (the default threshold, zero,
    // would hand it back at every stream synchronisation)
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = pool;
    return pool;
}

cudaError_t ctx_alloc(cfpq_ctx *c, void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, c->pool, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        cudaMemPoolTrimTo(c->pool, 0);
        e = cudaMallocFromPoolAsync(p, bytes, c->pool, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
    }
    return e;
}

void ctx_free(cfpq_ctx *c, void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

void free_ctx_device(cfpq_ctx *c) {
    // A context of cfpq_create may still have work in flight on a caller's stream or on its
    // side streams: let it finish before its memory goes back to the pool (cudaFree used to
    // synchronise the device in the same way). A server's contexts are retired only after
    // their stream's work has completed.
    if (!c->pooled) cudaDeviceSynchronize();
    tensor_release(c);
    worklist_release(c);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
    void *ptrs[] = {c->d_arena, c->d_triples, c->d_tc_work, c->d_lens, c->d_TTn};
    for (void *p : ptrs) ctx_free(c, p, c->stream);
    for (auto e : c->prof_ev)
        if (e) cudaEventDestroy(e);
    c->prof_ev.clear();
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->stream && c->own_stream) cudaStreamDestroy(c->stream);
    if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
    if (c->aux2_stream) cudaStreamDestroy(c->aux2_stream);
    c->aux_stream = c->aux2_stream = nullptr;
}

void arm_deadline(cfpq_ctx *c, cudaStream_t s) {
    k_arm_deadline<<<1, 1, 0, s>>>(c->d_state, (unsigned long long)(c->timeout_s * 1e9));
}

// Clears the matrices and seeds them from the edges (Algorithm 1's initialisation).
int enqueue_reset_and_seed(cfpq_ctx *c, cudaStream_t s) {
    const size_t planes = (size_t)c->n_nt * c->plane * sizeof(uint32_t);
    if (!c->clean) {
        CK(cudaMemsetAsync(c->d_T, 0, planes, s));
        CK(cudaMemsetAsync(c->d_X0, 0, planes, s));
        CK(cudaMemsetAsync(c->d_X1, 0, planes, s));
        CK(cudaMemsetAsync(c->d_Tsum, 0, (size_t)c->n_nt * c->n_pad * c->SW * sizeof(uint32_t), s));
    }
    if (c->lengths) {  // T^T and its word summary are built pair by pair from here on
        const size_t sum = (size_t)c->n_nt * c->n_pad * c->SW * sizeof(uint32_t);
        CK(cudaMemsetAsync(c->d_TTsum, 0, sum, s));
        CK(cudaMemsetAsync(c->d_TT, 0, planes, s));
    }
    // the row bitmaps, the state and the deadline; on a converged context also the rows of T
    // that still hold bits
    const unsigned long long dt_ns = c->timeout_s > 0 ? (unsigned long long)(c->timeout_s * 1e9) : 0ull;
    k_reset<<<(uint32_t)((uint64_t)c->n_nt * c->W), 128, 0, s>>>(c->d_q, c->d_state0, dt_ns, c->clean ? 1 : 0);
    CK(cudaGetLastError());
    c->clean = false;
    c->fixed_launches = 2;  // k_reset and the seed
    const uint64_t work = std::max<uint64_t>(c->n_edges, (uint64_t)c->n_eps_rules * c->n);
    const uint32_t blocks = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(1, (work + 255) / 256), 148ull * 16);
    k_seed<<<blocks, 256, 0, s>>>(c->d_q);
    CK(cudaGetLastError());
    if (c->lengths) {
        const int rc = lengths_enqueue_seed(c, s);
        if (rc != CFPQ_OK) return rc;
        c->fixed_launches++;
    }
    if (c->any_gather) {  // the first execution's gather list
        int cpl;
        const uint32_t nch = gather_chunks(c->W, &cpl);
        const uint64_t items = (uint64_t)c->n_groups * ((c->n + 31) / 32);
        k_scan_rows<<<(uint32_t)((items + 255) / 256), 256, 0, s>>>(c->d_q, c->d_list, c->list_cap, nch);
        CK(cudaGetLastError());
        c->fixed_launches++;
    }
    bool any_tensor = false;
    for (int g = 0; g < c->n_groups; g++) any_tensor |= c->group_tensor[g] != 0;
    if (any_tensor) return enqueue_tensor_seed_transposes(c, s, &c->fixed_launches);
    return CFPQ_OK;
}

int read_status(cfpq_ctx *c, cudaStream_t s, unsigned *to_worklist) {
    DevState st;
    CK(cudaMemcpyAsync(&st, c->d_state, sizeof(st), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (to_worklist) *to_worklist = st.to_worklist;
    return apply_status(c, st);
}

int apply_status(cfpq_ctx *c, const DevState &st) {
    c->stats.iterations = (int64_t)st.iter;
    c->stats.new_bits = (int64_t)st.new_bits;
    c->stats.seed_bits = (int64_t)st.seed_bits;
    c->stats.tensor_products = (int64_t)st.tensor_products;
    c->stats.gather_products = (int64_t)st.gather_products;
    c->stats.dense_ops = 2.0 * (double)c->n_pad * (double)c->n_pad * (double)c->n_pad * (double)st.tensor_products;
    c->stats.n_pad = c->n_pad;
    c->stats.kernel_launches = c->fixed_launches + ((int64_t)st.iter - (int64_t)st.loop_execs) * c->iter_launches +
                               (int64_t)st.loop_launches;
    c->stats.product_bytes = 4.0 * (double)st.prof_words;
    c->stats.useful_ops = 2.0 * (double)st.useful_macs;
    c->stats.lengths_splits = (double)st.len_splits;
    c->stats.tensor_live_ops = kTcOpsPerStep * (double)st.tc_live_steps;
    int rc = CFPQ_OK;
    if (st.error == kErrIterLimit) rc = CFPQ_ERR_ITER_LIMIT;
    else if (st.error == kErrTimeout) rc = CFPQ_ERR_TIMEOUT;
    else if (st.error == kErrDevice) {
        rc = CFPQ_ERR_CUDA;
        if (getenv("CFPQ_VERBOSE"))
            fprintf(stderr,
                    "cfpq: a tensor product gave up: wait site %u, CTA %u, group %u, execution %u, %u tiles listed, "
                    "%u tiles claimed\n",
                    st.tc_diag[0], st.tc_diag[1] - 1u, st.tc_diag[2], st.tc_diag[3], st.tc_diag[4], st.tc_diag[5]);
    }
    c->stats.status = rc;
    return rc;
}

int ctx_init(cfpq_ctx *c, const cfpq_grammar_cnf *g, uint32_t n, const cfpq_edge *edges, size_t n_edges,
             const cfpq_options &o) {
    c->n = n;
    c->n_pad = (n + 255u) / 256u * 256u;
    c->W = c->n_pad / 32u;
    c->plane = (uint64_t)c->n_pad * c->W;
    c->lplane = (uint64_t)c->n_pad * c->n_pad;
    c->SW = ((c->W + 31u) / 32u + 3u) & ~3u;
    c->n_nt = g->n_nonterm;
    c->n_term = g->n_term;
    c->schedule_req = o.schedule;
    c->schedule = o.schedule == CFPQ_SCHED_AUTO ? CFPQ_SCHED_INPLACE : o.schedule;  // single solves
    c->path = o.path;
    c->lengths = o.lengths != 0;
    c->dense_tensor = o.dense_tensor != 0;
    c->tensor_kind = o.tensor_kind == CFPQ_TENSOR_FP8 ? CFPQ_TENSOR_FP8 : CFPQ_TENSOR_FP4;
    c->block = o.row_begin != 0 || o.row_end != 0;
    c->row0 = c->block ? o.row_begin : 0u;
    c->row1 = (!c->block || o.row_end == n) ? c->n_pad : o.row_end;
    if (c->block) {
        // a row block of a sharded solve: Algorithm 1's Jacobi loop body, on a matrix path
        if (o.schedule == CFPQ_SCHED_INPLACE || o.path == CFPQ_PATH_WORKLIST || c->lengths)
            return CFPQ_ERR_UNSUPPORTED;
        c->schedule = CFPQ_SCHED_JACOBI;
    }
    if (c->lengths) {
        // the lengths come from the matrices before each loop execution: Jacobi schedule only
        if (o.schedule == CFPQ_SCHED_INPLACE || o.path == CFPQ_PATH_WORKLIST) return CFPQ_ERR_UNSUPPORTED;
        c->schedule = CFPQ_SCHED_JACOBI;
    }
    c->use_graph = o.use_graph;
    c->profile = o.profile;
    c->timeout_s = o.timeout_s;
    const double bound = (double)n * (double)n * (double)g->n_nonterm + 1.0;
    c->max_iter = o.max_iter > 0 ? (uint64_t)o.max_iter : (bound > 1.8e19 ? ~0ull : (uint64_t)bound);
    // productions: dedupe, group by left-hand side
    std::vector<Rule> rules;
    for (int i = 0; i < g->n_binary; i++) rules.push_back({g->binary[i].lhs, g->binary[i].b, g->binary[i].c, 0});
    std::sort(rules.begin(), rules.end(), [](const Rule &x, const Rule &y) {
        if (x.lhs != y.lhs) return x.lhs < y.lhs;
        if (x.b != y.b) return x.b < y.b;
        return x.c < y.c;
    });
    rules.erase(std::unique(rules.begin(), rules.end(),
                            [](const Rule &x, const Rule &y) { return x.lhs == y.lhs && x.b == y.b && x.c == y.c; }),
                rules.end());
    std::vector<int32_t> gstart;
    for (size_t i = 0; i < rules.size(); i++)
        if (i == 0 || rules[i].lhs != rules[i - 1].lhs) gstart.push_back((int32_t)i);
    gstart.push_back((int32_t)rules.size());
    c->n_groups = (int)gstart.size() - 1;
    c->nt_dynamic.assign(g->n_nonterm, 0);
    for (const Rule &r : rules) c->nt_dynamic[r.lhs] = 1;
    c->rules = rules;
    c->gstart = gstart;
    if (c->lengths && !lengths_rules_ok(c)) return CFPQ_ERR_UNSUPPORTED;
    std::vector<int2> unary;
    for (int i = 0; i < g->n_unary; i++) unary.push_back(make_int2(g->unary[i].lhs, g->unary[i].term));
    std::vector<int32_t> eps(g->eps_lhs, g->eps_lhs + g->n_eps);
    std::sort(eps.begin(), eps.end());
    eps.erase(std::unique(eps.begin(), eps.end()), eps.end());
    c->n_unary = (int)unary.size();
    c->n_eps_rules = (int)eps.size();
    c->h_unary = unary;
    c->h_eps = eps;
    c->n_edges = n_edges;
    c->group_tensor.assign(std::max(1, c->n_groups), 0);
    if (c->path == CFPQ_PATH_TENSOR) {
        if (!tensor_path_available()) return CFPQ_ERR_UNSUPPORTED;
        c->group_tensor.assign(std::max(1, c->n_groups), 1);
    }
    c->auto_mixed = c->path == CFPQ_PATH_AUTO && c->n_groups > 0 && tensor_path_available();
    c->allow_switch = c->path == CFPQ_PATH_AUTO && c->n_groups > 0 && c->schedule != CFPQ_SCHED_JACOBI;
    c->any_gather = c->n_groups > 0 && c->path != CFPQ_PATH_TENSOR && c->path != CFPQ_PATH_WORKLIST;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            c->sms = sms;
        cudaGetLastError();
    }
    {
        int cpl;
        const uint64_t slots = c->any_gather ? (uint64_t)c->n_groups * c->n * gather_chunks(c->W, &cpl) : 0;
        if (slots > 0xFFFFFFFFull) return CFPQ_ERR_INVALID;
        c->list_cap = (uint32_t)slots;
        if (c->any_gather) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const void *fn = cpl == 1 ? (const void *)k_gather_list<1> : cpl == 2 ? (const void *)k_gather_list<2>
                           : cpl == 4 ? (const void *)k_gather_list<4> : (const void *)k_gather_list<8>;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
            c->gather_grid = std::max(1, sms) * per_sm;
            // the persistent loop of gather-only executions: every block resident at once. Small
            // problems take fewer blocks (a barrier then gathers fewer arrivals): one per SM up to
            // n = 4096, two up to 8192, else all that fit (measured on hierarchy queries, n = 512 ..
            // 16384: one per SM is 7 % faster than three at n <= 2048, three 27 % faster than one
            // at 16384)
            int coop = 0, loop_per_sm = 0;
            const void *lf = c->lengths
                                 ? (cpl == 1 ? (const void *)k_gather_loop<1, true> : cpl == 2 ? (const void *)k_gather_loop<2, true>
                                    : cpl == 4 ? (const void *)k_gather_loop<4, true> : (const void *)k_gather_loop<8, true>)
                                 : (cpl == 1 ? (const void *)k_gather_loop<1, false> : cpl == 2 ? (const void *)k_gather_loop<2, false>
                                    : cpl == 4 ? (const void *)k_gather_loop<4, false> : (const void *)k_gather_loop<8, false>);
            c->loop_grid = 0;
            if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&loop_per_sm, lf, 256, 0) == cudaSuccess && loop_per_sm > 0)
                c->loop_grid = std::max(1, sms) * std::min(loop_per_sm, n <= 4096u ? 1 : n <= 8192u ? 2 : loop_per_sm);
            cudaGetLastError();
        }
    }

    if (!c->pooled) {
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    c->last_stream = c->stream;
    CK(cudaEventCreate(&c->ev0));
    CK(cudaEventCreate(&c->ev1));
    if (c->profile) {
        c->prof_ev.assign(2 * (c->n_groups + 2), nullptr);
        for (auto &e : c->prof_ev) CK(cudaEventCreate(&e));
    }
    // one arena for every buffer of the query (one allocation, one free). The batched
    // launch clears T, X0, X1 as one span and R0, R1, Trow as another: keep each run of
    // parts adjacent and in this order
    const size_t planes = (size_t)c->n_nt * c->plane * sizeof(uint32_t);
    const size_t rowsz = (size_t)c->n_nt * c->W * sizeof(uint32_t);
    const size_t cells = (size_t)c->n_nt * c->n_pad;  // (non-terminal, row) extraction cells
    const bool want_tt = (c->path == CFPQ_PATH_WORKLIST) || c->allow_switch || c->lengths ||
                         ((c->path == CFPQ_PATH_AUTO || c->path == CFPQ_PATH_TENSOR) && tensor_path_available());
    // tile occupancy for the tensor products (unless dense products were asked for)
    const bool occ = !c->dense_tensor && (c->path == CFPQ_PATH_AUTO || c->path == CFPQ_PATH_TENSOR) &&
                     tensor_path_available() && c->n_groups > 0;
    const size_t swk = ((c->n_pad / 128) + 31) / 32;
    struct Part { void **dst; size_t bytes; };
    const Part parts[] = {
        {(void **)&c->d_T, planes}, {(void **)&c->d_X0, planes}, {(void **)&c->d_X1, planes},
        {(void **)&c->d_TT, want_tt ? planes : 0}, {(void **)&c->d_R0, rowsz}, {(void **)&c->d_R1, rowsz},
        {(void **)&c->d_Trow, rowsz}, {(void **)&c->d_rules, rules.size() * sizeof(Rule)},
        {(void **)&c->d_gstart, gstart.size() * sizeof(int32_t)}, {(void **)&c->d_unary, unary.size() * sizeof(int2)},
        {(void **)&c->d_nt_rules, (size_t)c->n_nt * sizeof(int2)},
        {(void **)&c->d_eps, eps.size() * sizeof(int32_t)}, {(void **)&c->d_edges, n_edges * sizeof(cfpq_edge)},
        {(void **)&c->d_state, sizeof(DevState)}, {(void **)&c->d_state0, sizeof(DevState)},
        {(void **)&c->d_q, sizeof(QDesc)},
        {(void **)&c->d_counts, cells * sizeof(uint32_t)}, {(void **)&c->d_offsets, cells * sizeof(uint64_t)},
        {(void **)&c->d_block_sums, (kScanMaxBlocks + 1) * sizeof(unsigned long long)},
        {(void **)&c->d_nt_off, (size_t)(c->n_nt + 1) * sizeof(unsigned long long)},
        {(void **)&c->d_total, sizeof(unsigned long long)},
        {(void **)&c->d_choice, sizeof(cudaGraphConditionalHandle) * (kMaxNT + 2)},
        {(void **)&c->d_list, (size_t)c->list_cap * sizeof(uint32_t)},
        {(void **)&c->d_colcnt, c->profile ? sizeof(uint32_t) * c->n_pad : 0},
        {(void **)&c->d_L, c->lengths ? (size_t)c->n_nt * c->n_pad * c->n_pad * sizeof(uint32_t) : 0},
        {(void **)&c->d_Wit, c->lengths ? (size_t)c->n_nt * c->n_pad * c->n_pad * sizeof(uint32_t) : 0},
        {(void **)&c->d_Tsum, (size_t)c->n_nt * c->n_pad * c->SW * sizeof(uint32_t)},
        {(void **)&c->d_TTsum, c->lengths ? (size_t)c->n_nt * c->n_pad * c->SW * sizeof(uint32_t) : 0},
        {(void **)&c->d_occA, occ ? (size_t)c->n_nt * (c->n_pad / 128) * swk * sizeof(uint32_t) : 0},
        {(void **)&c->d_occB, occ ? (size_t)c->n_nt * (c->n_pad / 256) * swk * sizeof(uint32_t) : 0},
        {(void **)&c->d_occCA, occ ? (size_t)c->n_nt * (c->n_pad / 128) * sizeof(uint32_t) : 0},
        {(void **)&c->d_occCB, occ ? (size_t)c->n_nt * (c->n_pad / 128) * sizeof(uint32_t) : 0},
        {(void **)&c->d_occKnown, occ ? (size_t)c->n_nt * sizeof(uint32_t) : 0},
        {(void **)&c->d_tile_list, occ ? (size_t)(c->n_pad / 256) * (c->n_pad / 128) * 8 : 0}};
    size_t arena = 0;
    for (const Part &pt : parts) arena += (pt.bytes + 255) / 256 * 256;
    if (!c->pool) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        c->pool = library_pool(dev);
        if (!c->pool) return CFPQ_ERR_UNSUPPORTED;
    }
    {
        void *arena_p = nullptr;
        const cudaError_t e = ctx_alloc(c, &arena_p, arena, c->stream);
        if (e == cudaErrorMemoryAllocation) return CFPQ_ERR_NOMEM;
        if (e != cudaSuccess) return CFPQ_ERR_CUDA;
        c->d_arena = arena_p;
    }
    {
        char *p = static_cast<char *>(c->d_arena);
        for (const Part &pt : parts) {
            *pt.dst = pt.bytes ? p : nullptr;
            p += (pt.bytes + 255) / 256 * 256;
        }
    }
    // copies are stream-ordered after the (possibly stream-ordered) allocations; the host
    // sources are pageable, so each call returns once its source has been staged
    cudaStream_t cs = c->stream;
    if (occ) {
        // tile occupancy starts empty, its counts zero: the occupancy passes keep the two
        // consistent by counting the bits they flip
        const uint32_t swk2 = ((c->n_pad / 128) + 31) / 32;
        CK(cudaMemsetAsync(c->d_occA, 0, (size_t)c->n_nt * (c->n_pad / 128) * swk2 * sizeof(uint32_t), cs));
        CK(cudaMemsetAsync(c->d_occB, 0, (size_t)c->n_nt * (c->n_pad / 256) * swk2 * sizeof(uint32_t), cs));
        CK(cudaMemsetAsync(c->d_occCA, 0, (size_t)c->n_nt * (c->n_pad / 128) * sizeof(uint32_t), cs));
        CK(cudaMemsetAsync(c->d_occCB, 0, (size_t)c->n_nt * (c->n_pad / 128) * sizeof(uint32_t), cs));
        CK(cudaMemsetAsync(c->d_occKnown, 0, (size_t)c->n_nt * sizeof(uint32_t), cs));
    }
    if (!rules.empty())
        CK(cudaMemcpyAsync(c->d_rules, rules.data(), rules.size() * sizeof(Rule), cudaMemcpyHostToDevice, cs));
    CK(cudaMemcpyAsync(c->d_gstart, gstart.data(), gstart.size() * sizeof(int32_t), cudaMemcpyHostToDevice, cs));
    c->h_nt_rules.assign(c->n_nt, make_int2(-1, -1));
    for (int gr = 0; gr < c->n_groups; gr++) c->h_nt_rules[rules[gstart[gr]].lhs] = make_int2(gstart[gr], gstart[gr + 1]);
    CK(cudaMemcpyAsync(c->d_nt_rules, c->h_nt_rules.data(), c->n_nt * sizeof(int2), cudaMemcpyHostToDevice, cs));
    if (!unary.empty())
        CK(cudaMemcpyAsync(c->d_unary, unary.data(), unary.size() * sizeof(int2), cudaMemcpyHostToDevice, cs));
    if (!eps.empty()) CK(cudaMemcpyAsync(c->d_eps, eps.data(), eps.size() * sizeof(int32_t), cudaMemcpyHostToDevice, cs));
    if (n_edges) CK(cudaMemcpyAsync(c->d_edges, edges, n_edges * sizeof(cfpq_edge), cudaMemcpyHostToDevice, cs));
    QDesc q;
    memset(&q, 0, sizeof(q));
    q.n = n;
    q.n_pad = c->n_pad;
    q.W = c->W;
    q.n_nt = c->n_nt;
    q.n_rules = (int32_t)rules.size();
    q.n_groups = c->n_groups;
    q.schedule = c->schedule;
    q.profile = c->profile;
    q.allow_switch = c->allow_switch ? 1 : 0;
    q.n_unary = c->n_unary;
    q.n_eps = c->n_eps_rules;
    q.plane = c->plane;
    q.n_edges = n_edges;
    q.T = c->d_T;
    q.TT = c->d_TT;
    q.X0 = c->d_X0;
    q.X1 = c->d_X1;
    q.R0 = c->d_R0;
    q.R1 = c->d_R1;
    q.Trow = c->d_Trow;
    q.occA = c->d_occA;
    q.occB = c->d_occB;
    q.occCA = c->d_occCA;
    q.occCB = c->d_occCB;
    q.occKnown = c->d_occKnown;
    q.tensor_kind = c->tensor_kind;
    q.KS = c->n_pad / 128;
    q.SWK = (q.KS + 31) / 32;
    q.Tsum = c->d_Tsum;
    q.TTsum = c->d_TTsum;
    q.SW = c->SW;
    q.row0 = c->row0;
    q.row1 = c->row1;
    q.rules = c->d_rules;
    q.gstart = c->d_gstart;
    q.nt_rules = c->d_nt_rules;
    q.unary = c->d_unary;
    q.eps = c->d_eps;
    q.edges = c->d_edges;
    q.st = c->d_state;
    c->hq = q;
    CK(cudaMemcpyAsync(c->d_q, &q, sizeof(q), cudaMemcpyHostToDevice, cs));
    {
        // the state every solve starts from: no executions yet, every transpose and tile
        // occupancy to be built, the groups' product kinds (the loop's tail plans the rest)
        DevState st0;
        memset(&st0, 0, sizeof(st0));
        st0.max_iter = c->max_iter;
        for (int a = 0; a < c->n_nt; a++) st0.dirty[a] = st0.occ_now[a] = 1u;
        for (int g = 0; g < c->n_groups && g < kMaxNT; g++) st0.use_tensor[g] = c->group_tensor[g] ? 1u : 0u;
        CK(cudaMemcpyAsync(c->d_state0, &st0, sizeof(st0), cudaMemcpyHostToDevice, cs));
    }
    if (c->path == CFPQ_PATH_WORKLIST) return worklist_setup(c, false);
    // the set-up above ran on the context's stream, and a solve may run on any stream the
    // caller names: finish it here (a server's contexts share the server's stream)
    if (!c->pooled) CK(cudaStreamSynchronize(cs));
    return CFPQ_OK;
}

size_t query_footprint(uint32_t n, int n_nt, size_t n_edges, int n_rules, bool tensor) {
    const size_t n_pad = (n + 255u) / 256u * 256u;
    const size_t plane = n_pad * (n_pad / 32) * 4;
    const size_t planes = (tensor ? 4 : 3) * (size_t)n_nt * plane;
    const size_t rows = 3 * (size_t)n_nt * (n_pad / 8);
    const size_t list = (size_t)n_rules * n * ((n_pad / 32 + 255) / 256) * 4;  // gather items (at most)
    const size_t misc = n_edges * sizeof(cfpq_edge) + n_pad * 12 + (size_t)n_rules * 32 + 64 * 1024 + list;
    return planes + rows + misc;
}

int validate_inputs(const cfpq_grammar_cnf *g, uint32_t n, const cfpq_edge *edges, size_t n_edges,
                    const cfpq_options *opt) {
    if (!g || n == 0 || n > CFPQ_MAX_NODES) return CFPQ_ERR_INVALID;
    if (g->n_nonterm <= 0 || g->n_nonterm > CFPQ_MAX_NONTERM || g->n_term < 0) return CFPQ_ERR_INVALID;
    if (g->n_unary < 0 || g->n_binary < 0 || g->n_eps < 0) return CFPQ_ERR_INVALID;
    if ((g->n_unary > 0 && !g->unary) || (g->n_binary > 0 && !g->binary) || (g->n_eps > 0 && !g->eps_lhs))
        return CFPQ_ERR_INVALID;
    if (n_edges > 0 && !edges) return CFPQ_ERR_INVALID;
    for (int i = 0; i < g->n_unary; i++)
        if (g->unary[i].lhs < 0 || g->unary[i].lhs >= g->n_nonterm || g->unary[i].term < 0 ||
            g->unary[i].term >= g->n_term)
            return CFPQ_ERR_INVALID;
    for (int i = 0; i < g->n_binary; i++) {
        const cfpq_rule2 r = g->binary[i];
        if (r.lhs < 0 || r.lhs >= g->n_nonterm || r.b < 0 || r.b >= g->n_nonterm || r.c < 0 || r.c >= g->n_nonterm)
            return CFPQ_ERR_INVALID;
    }
    for (int i = 0; i < g->n_eps; i++)
        if (g->eps_lhs[i] < 0 || g->eps_lhs[i] >= g->n_nonterm) return CFPQ_ERR_INVALID;
    for (size_t e = 0; e < n_edges; e++)
        if (edges[e].src >= n || edges[e].dst >= n || edges[e].label < 0 || edges[e].label >= g->n_term)
            return CFPQ_ERR_INVALID;
    if (opt) {
        if (opt->schedule != CFPQ_SCHED_INPLACE && opt->schedule != CFPQ_SCHED_JACOBI &&
            opt->schedule != CFPQ_SCHED_AUTO)
            return CFPQ_ERR_INVALID;
        if (opt->path < CFPQ_PATH_AUTO || opt->path > CFPQ_PATH_WORKLIST) return CFPQ_ERR_INVALID;
        if ((opt->lengths != 0 && opt->lengths != 1) || (opt->dense_tensor != 0 && opt->dense_tensor != 1))
            return CFPQ_ERR_INVALID;
        if (opt->tensor_kind < CFPQ_TENSOR_AUTO || opt->tensor_kind > CFPQ_TENSOR_FP4) return CFPQ_ERR_INVALID;
        if (opt->row_begin != 0 || opt->row_end != 0) {  // a row block: 256-aligned ends inside [0, n]
            if (opt->row_begin % 256u != 0 || opt->row_begin >= opt->row_end || opt->row_end > n ||
                (opt->row_end % 256u != 0 && opt->row_end != n))
                return CFPQ_ERR_INVALID;
        }
    }
    return CFPQ_OK;
}

int ctx_create_pooled(const cfpq_grammar_cnf *g, uint32_t n, const cfpq_edge *edges, size_t n_edges,
                      const cfpq_options &o, cudaStream_t pool_stream, cfpq_ctx **out) {
    cfpq_ctx *c = new (std::nothrow) cfpq_ctx();
    if (!c) return CFPQ_ERR_NOMEM;
    c->pooled = true;
    c->stream = pool_stream;
    c->own_stream = false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetDefaultMemPool(&c->pool, dev) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return CFPQ_ERR_CUDA;
    }
    const int rc = ctx_init(c, g, n, edges, n_edges, o);
    if (rc != CFPQ_OK) {
        free_ctx_device(c);
        delete c;
        return rc;
    }
    *out = c;
    return CFPQ_OK;
}

void ctx_destroy(cfpq_ctx *c) {
    if (!c) return;
    free_ctx_device(c);
    delete c;
}

int run_loop(cfpq_ctx *c, cudaStream_t s) {
    if (c->n_groups == 0) {
        // no binary productions: one execution of the loop body finds nothing new
        k_tail<<<1, 1024, 0, s>>>(c->d_q, 0, 0, nullptr, 0);
        c->iter_launches = 1;
        CK(cudaGetLastError());
        return CFPQ_OK;
    }
    if (c->use_graph && !c->profile) {
        const int rc = build_graph(c);
        if (rc != CFPQ_OK) return rc;
        CK(cudaGraphLaunch(c->graph_exec, s));
        return CFPQ_OK;
    }
    for (;;) {
        int rc = enqueue_iteration(c, s, 0, 0);
        if (rc != CFPQ_OK) return rc;
        unsigned cont = 0;
        CK(cudaMemcpyAsync(&cont, &c->d_state->cont, sizeof(cont), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (c->profile && (rc = collect_profile(c)) != CFPQ_OK) return rc;
        if (!cont) break;
    }
    return CFPQ_OK;
}

static int count_rows_and_scan(cfpq_ctx *c, int32_t A, cudaStream_t s, unsigned long long *total) {
    k_count_rows<<<row_warp_blocks(c->n_pad), 256, 0, s>>>(c->d_q, A, c->d_counts);
    k_scan<<<1, 1024, 0, s>>>(c->d_counts, c->d_offsets, c->n_pad, c->d_total);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(total, c->d_total, sizeof(*total), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return CFPQ_OK;
}

static int emit(cfpq_ctx *c, int32_t A, cfpq_triple *dev_out, cudaStream_t s) {
    k_emit<<<row_warp_blocks(c->n_pad), 256, 0, s>>>(c->d_q, A, c->d_offsets, c->d_counts, dev_out);
    CK(cudaGetLastError());
    return CFPQ_OK;
}

}  // namespace cfpq

extern "C" int cfpq_create(const cfpq_grammar_cnf *g, uint32_t n, const cfpq_edge *edges, size_t n_edges,
                           const cfpq_options *opt, cfpq_ctx **out) {
    if (!out) return CFPQ_ERR_INVALID;
    const int vrc = validate_inputs(g, n, edges, n_edges, opt);
    if (vrc != CFPQ_OK) return vrc;
    cfpq_options o;
    cfpq_options_default(&o);
    if (opt) o = *opt;

    cfpq_ctx *c = new (std::nothrow) cfpq_ctx();
    if (!c) return CFPQ_ERR_NOMEM;
    const int rc = ctx_init(c, g, n, edges, n_edges, o);
    if (rc != CFPQ_OK) {
        free_ctx_device(c);
        delete c;
        return rc;
    }
    *out = c;
    return CFPQ_OK;
}

// The asynchronous part of a solve: the matrix initialisation and the loop (a graph launch
// or the host-driven loop) enqueued on s, the end event recorded.
int cfpq::solve_begin(cfpq_ctx *c, cudaStream_t s) {
    c->solved = false;
    c->last_stream = s;
    c->stats.product_ms = c->stats.tensor_ms = c->stats.lengths_ms = 0.0;
    c->stats.product_launches = c->stats.tensor_launches = c->stats.lengths_launches = 0;
    CK(cudaEventRecord(c->ev0, s));
    int rc = enqueue_reset_and_seed(c, s);
    if (rc != CFPQ_OK) return rc;
    rc = c->path == CFPQ_PATH_WORKLIST ? worklist_run(c, s) : run_loop(c, s);
    if (rc != CFPQ_OK) return rc;
    CK(cudaEventRecord(c->ev1, s));
    return CFPQ_OK;
}

// The rest of a solve begun on s: the status (waits for the loop), the hand-over to the
// worklist path where the loop asked for it, and the statistics.
int cfpq::solve_end(cfpq_ctx *c, cudaStream_t s) {
    unsigned to_wl = 0;
    int rc = read_status(c, s, &to_wl);
    if (rc == CFPQ_ERR_CUDA) return rc;
    c->switched = false;
    if (rc == CFPQ_OK && c->allow_switch) {
        // the loop stopped after a long run of tiny deltas: the worklist path finishes the
        // closure from the current delta (same least fixpoint)
        if (to_wl) {
            if (!c->h_wl && (rc = worklist_setup(c, true)) != CFPQ_OK) return rc;
            const int64_t loops = c->stats.iterations;
            if ((rc = worklist_run(c, s, true)) != CFPQ_OK) return rc;
            CK(cudaEventRecord(c->ev1, s));
            rc = read_status(c, s);
            if (rc == CFPQ_ERR_CUDA) return rc;
            c->stats.iterations = loops;  // loop executions before the hand-over
            c->switched = true;
        }
    }
    // a loop that converged leaves both delta planes zero (each execution clears the delta it
    // read, the last one adds nothing); the worklist path and an interrupted loop do not
    c->clean = rc == CFPQ_OK && !c->switched && c->path != CFPQ_PATH_WORKLIST && c->n_groups > 0;
    // an interrupted loop can go on from where it stopped (cfpq_resume)
    c->resumable = (rc == CFPQ_ERR_ITER_LIMIT || rc == CFPQ_ERR_TIMEOUT) && !c->switched;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    c->stats.solve_ms = ms;
    c->stats.schedule = c->schedule;
    c->stats.gather_cpl = 0;
    c->solved = true;
    return rc;
}

extern "C" int cfpq_solve(cfpq_ctx *c, void *stream) {
    if (!c || c->block) return CFPQ_ERR_INVALID;  // a row block is solved with the cfpq_block_* calls
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const int rc = solve_begin(c, s);
    if (rc != CFPQ_OK) return rc;
    return solve_end(c, s);
}

extern "C" int cfpq_block_start(cfpq_ctx *c, void *stream) {
    if (!c || !c->block) return CFPQ_ERR_INVALID;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    c->solved = false;
    c->last_stream = s;
    c->stats.product_ms = c->stats.tensor_ms = c->stats.lengths_ms = 0.0;
    c->stats.product_launches = c->stats.tensor_launches = c->stats.lengths_launches = 0;
    CK(cudaEventRecord(c->ev0, s));
    const int rc = enqueue_reset_and_seed(c, s);
    if (rc != CFPQ_OK) return rc;
    c->block_started = true;
    return CFPQ_OK;
}

extern "C" int cfpq_block_products(cfpq_ctx *c, void *stream) {
    if (!c || !c->block) return CFPQ_ERR_INVALID;
    if (!c->block_started) return CFPQ_ERR_NOT_SOLVED;
    if (c->n_groups == 0) return CFPQ_OK;  // no binary productions: nothing to multiply
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    c->last_stream = s;
    c->iter_launches = 0;
    return enqueue_products(c, s, 0);
}

extern "C" int cfpq_block_export(cfpq_ctx *c, uint32_t *buf, size_t cap_words, size_t *words, void *stream) {
    if (!c || !c->block || !words || (!buf && cap_words > 0)) return CFPQ_ERR_INVALID;
    if (!c->block_started) return CFPQ_ERR_NOT_SOLVED;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const uint64_t rec_words = 2u + c->W;
    unsigned long long records = 0;
    if (c->n_groups > 0) {
        CK(cudaMemsetAsync(&c->d_state->block_records, 0, sizeof(unsigned long long), s));
        const uint32_t units = (uint32_t)((uint64_t)c->n_nt * ((std::min(c->row1, c->n) + 31u) / 32u - c->row0 / 32u));
        k_block_pack<<<std::min<uint32_t>(std::max<uint32_t>(1u, (units + 7u) / 8u), 8u * (uint32_t)c->sms), 256, 0,
                       s>>>(c->d_q, buf, buf ? (uint64_t)(cap_words / rec_words) : 0ull);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&records, &c->d_state->block_records, sizeof(records), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    *words = (size_t)(records * rec_words);
    return records * rec_words > cap_words ? CFPQ_ERR_BUFFER : CFPQ_OK;
}

extern "C" int cfpq_block_import(cfpq_ctx *c, const uint32_t *buf, size_t words, void *stream) {
    if (!c || !c->block || (!buf && words > 0)) return CFPQ_ERR_INVALID;
    if (!c->block_started) return CFPQ_ERR_NOT_SOLVED;
    const uint64_t rec_words = 2u + c->W;
    if (words % rec_words != 0) return CFPQ_ERR_INVALID;
    if (words == 0 || c->n_groups == 0) return CFPQ_OK;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const uint64_t n_records = words / rec_words;
    k_block_import<<<(uint32_t)std::min<uint64_t>((n_records + 7u) / 8u, 8ull * (uint64_t)c->sms), 256, 0, s>>>(
        c->d_q, buf, n_records);
    CK(cudaGetLastError());
    return CFPQ_OK;
}

extern "C" int cfpq_block_finish(cfpq_ctx *c, void *stream, int32_t *changed) {
    if (!c || !c->block || !changed) return CFPQ_ERR_INVALID;
    if (!c->block_started) return CFPQ_ERR_NOT_SOLVED;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    int rc;
    if (c->n_groups == 0) {
        k_tail<<<1, 1024, 0, s>>>(c->d_q, 0, 0, nullptr, 0);
        c->iter_launches = 1;
        CK(cudaGetLastError());
    } else if ((rc = enqueue_iteration_end(c, s, 0, 0)) != CFPQ_OK) {
        return rc;
    }
    CK(cudaEventRecord(c->ev1, s));
    DevState st;
    CK(cudaMemcpyAsync(&st, c->d_state, sizeof(st), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    rc = apply_status(c, st);
    if (st.block_bad) rc = CFPQ_ERR_INVALID;
    *changed = (rc == CFPQ_OK && st.cont) ? 1 : 0;
    if (!*changed) {
        // the solve ended (converged, or a limit or an error): the relations are readable
        c->block_started = false;
        c->solved = true;
        c->clean = rc == CFPQ_OK;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        c->stats.solve_ms = ms;
        c->stats.schedule = c->schedule;
    }
    return rc;
}

extern "C" int cfpq_count(cfpq_ctx *c, int32_t A, size_t *count) {
    if (!c || !count || A < 0 || A >= c->n_nt) return CFPQ_ERR_INVALID;
    if (!c->solved) return CFPQ_ERR_NOT_SOLVED;
    unsigned long long total = 0;
    const int rc = count_rows_and_scan(c, A, c->last_stream, &total);
    if (rc != CFPQ_OK) return rc;
    *count = (size_t)total;
    return CFPQ_OK;
}

extern "C" int cfpq_get_device(cfpq_ctx *c, int32_t A, cfpq_triple *buf, size_t cap, size_t *count) {
    if (!c || !count || A < 0 || A >= c->n_nt) return CFPQ_ERR_INVALID;
    if (!c->solved) return CFPQ_ERR_NOT_SOLVED;
    cudaStream_t s = c->last_stream;
    unsigned long long total = 0;
    const int rc = count_rows_and_scan(c, A, s, &total);
    if (rc != CFPQ_OK) return rc;
    *count = (size_t)total;
    if (!buf) return CFPQ_OK;
    if (cap < total) return CFPQ_ERR_BUFFER;
    if (total == 0) return CFPQ_OK;
    return emit(c, A, buf, s);
}

namespace cfpq {

// Grows the context's device triples buffer to hold `total` triples.
int ensure_triples(cfpq_ctx *c, size_t total, cudaStream_t s) {
    if (c->triples_cap >= total) return CFPQ_OK;
    ctx_free(c, c->d_triples, s);
    c->d_triples = nullptr;
    c->triples_cap = 0;
    void *p = nullptr;
    if (ctx_alloc(c, &p, total * sizeof(cfpq_triple), s) != cudaSuccess) return CFPQ_ERR_NOMEM;
    c->d_triples = static_cast<cfpq_triple *>(p);
    c->triples_cap = total;
    return CFPQ_OK;
}

}  // namespace cfpq

extern "C" int cfpq_get(cfpq_ctx *c, int32_t A, cfpq_triple *buf, size_t cap, size_t *count) {
    if (!c || !count || A < 0 || A >= c->n_nt) return CFPQ_ERR_INVALID;
    if (!c->solved) return CFPQ_ERR_NOT_SOLVED;
    cudaStream_t s = c->last_stream;
    unsigned long long total = 0;
    int rc = count_rows_and_scan(c, A, s, &total);
    if (rc != CFPQ_OK) return rc;
    *count = (size_t)total;
    if (!buf) return CFPQ_OK;
    if (cap < total) return CFPQ_ERR_BUFFER;
    if (total == 0) return CFPQ_OK;
    if ((rc = ensure_triples(c, total, s)) != CFPQ_OK) return rc;
    if ((rc = emit(c, A, c->d_triples, s)) != CFPQ_OK) return rc;
    CK(cudaMemcpyAsync(buf, c->d_triples, total * sizeof(cfpq_triple), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return CFPQ_OK;
}

namespace cfpq {

// Counts every relation and returns the first triple of each non-terminal (n_nt + 1
// entries, the last = total). One synchronisation.
// The counts, the offsets of every (non-terminal, row) cell and the per-non-terminal offsets
// (n_nt + 1 of them, copied to host memory h_nt_off when the stream reaches the copy; page-
// locked memory keeps the copy asynchronous), without waiting.
int count_all_enqueue(cfpq_ctx *c, cudaStream_t s, unsigned long long *h_nt_off) {
    const uint64_t cells = (uint64_t)c->n_nt * c->n_pad;
    const int nb = (int)((cells + kScanSeg - 1) / kScanSeg);
    k_count_all<<<row_warp_blocks(cells), 256, 0, s>>>(c->d_q, c->d_counts);
    k_scan_blocks<<<nb, 1024, 0, s>>>(c->d_counts, cells, c->d_block_sums);
    k_scan_bsums<<<1, 1024, 0, s>>>(c->d_block_sums, nb, c->d_total);
    k_scan_apply<<<nb, 1024, 0, s>>>(c->d_counts, cells, c->d_block_sums, c->d_offsets);
    k_nt_offsets<<<1, 96, 0, s>>>(c->d_q, c->d_offsets, c->d_total, c->d_nt_off);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h_nt_off, c->d_nt_off, (c->n_nt + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    return CFPQ_OK;
}

int count_all(cfpq_ctx *c, cudaStream_t s, std::vector<unsigned long long> &nt_off) {
    nt_off.assign(c->n_nt + 1, 0);
    const int rc = count_all_enqueue(c, s, nt_off.data());
    if (rc != CFPQ_OK) return rc;
    CK(cudaStreamSynchronize(s));
    return CFPQ_OK;
}

// Emits every relation (after count_all) into device memory `out`.
int emit_all(cfpq_ctx *c, cfpq_triple *out, cudaStream_t s) {
    const uint64_t cells = (uint64_t)c->n_nt * c->n_pad;
    k_emit_all<<<row_warp_blocks(cells), 256, 0, s>>>(c->d_q, c->d_offsets, c->d_counts, out);
    CK(cudaGetLastError());
    return CFPQ_OK;
}

// Every relation copied to host memory, one vector per non-terminal. Two synchronisations.
int extract_all_host(cfpq_ctx *c, std::vector<std::vector<cfpq_triple>> &out) {
    cudaStream_t s = c->last_stream;
    std::vector<unsigned long long> nt_off;
    int rc = count_all(c, s, nt_off);
    if (rc != CFPQ_OK) return rc;
    const size_t total = (size_t)nt_off[c->n_nt];
    out.assign(c->n_nt, {});
    if (total == 0) return CFPQ_OK;
    if ((rc = ensure_triples(c, total, s)) != CFPQ_OK) return rc;
    if ((rc = emit_all(c, c->d_triples, s)) != CFPQ_OK) return rc;
    std::vector<cfpq_triple> all(total);
    CK(cudaMemcpyAsync(all.data(), c->d_triples, total * sizeof(cfpq_triple), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int a = 0; a < c->n_nt; a++) out[a].assign(all.begin() + nt_off[a], all.begin() + nt_off[a + 1]);
    return CFPQ_OK;
}

}  // namespace cfpq

extern "C" int cfpq_get_all(cfpq_ctx *c, cfpq_triple *buf, size_t cap, size_t *count) {
    if (!c || !count) return CFPQ_ERR_INVALID;
    if (!c->solved) return CFPQ_ERR_NOT_SOLVED;
    cudaStream_t s = c->last_stream;
    std::vector<unsigned long long> nt_off;
    int rc = count_all(c, s, nt_off);
    if (rc != CFPQ_OK) return rc;
    const size_t total = (size_t)nt_off[c->n_nt];
    *count = total;
    if (!buf) return CFPQ_OK;
    if (cap < total) return CFPQ_ERR_BUFFER;
    if (total == 0) return CFPQ_OK;
    if ((rc = ensure_triples(c, total, s)) != CFPQ_OK) return rc;
    if ((rc = emit_all(c, c->d_triples, s)) != CFPQ_OK) return rc;
    CK(cudaMemcpyAsync(buf, c->d_triples, total * sizeof(cfpq_triple), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return CFPQ_OK;
}

extern "C" int cfpq_get_lengths(cfpq_ctx *c, int32_t A, cfpq_triple *buf, uint32_t *lengths, size_t cap,
                                size_t *count) {
    if (!c || !count || A < 0 || A >= c->n_nt || (!buf) != (!lengths)) return CFPQ_ERR_INVALID;
    if (!c->lengths) return CFPQ_ERR_UNSUPPORTED;
    if (!c->solved) return CFPQ_ERR_NOT_SOLVED;
    cudaStream_t s = c->last_stream;
    unsigned long long total = 0;
    int rc = count_rows_and_scan(c, A, s, &total);
    if (rc != CFPQ_OK) return rc;
    *count = (size_t)total;
    if (!buf) return CFPQ_OK;
    if (cap < total) return CFPQ_ERR_BUFFER;
    if (total == 0) return CFPQ_OK;
    if ((rc = ensure_triples(c, total, s)) != CFPQ_OK) return rc;
    if (c->lens_cap < total) {
        ctx_free(c, c->d_lens, s);
        c->d_lens = nullptr;
        c->lens_cap = 0;
        void *p = nullptr;
        if (ctx_alloc(c, &p, total * sizeof(uint32_t), s) != cudaSuccess) return CFPQ_ERR_NOMEM;
        c->d_lens = static_cast<uint32_t *>(p);
        c->lens_cap = total;
    }
    if ((rc = emit(c, A, c->d_triples, s)) != CFPQ_OK) return rc;
    if ((rc = lengths_of_triples(c, c->d_triples, total, c->d_lens, s)) != CFPQ_OK) return rc;
    CK(cudaMemcpyAsync(buf, c->d_triples, total * sizeof(cfpq_triple), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(lengths, c->d_lens, total * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return CFPQ_OK;
}

extern "C" int cfpq_get_path(cfpq_ctx *c, int32_t A, uint32_t m, uint32_t n, uint32_t *nodes, int32_t *labels,
                             size_t cap, size_t *len) {
    if (!c || !len || A < 0 || A >= c->n_nt || m >= c->n || n >= c->n || (!nodes) != (!labels)) return CFPQ_ERR_INVALID;
    if (!c->lengths) return CFPQ_ERR_UNSUPPORTED;
    if (!c->solved) return CFPQ_ERR_NOT_SOLVED;
    cudaStream_t s = c->last_stream;
    uint32_t word = 0, l = 0;
    CK(cudaMemcpyAsync(&word, c->d_T + (uint64_t)A * c->plane + (uint64_t)m * c->W + n / 32, sizeof(word),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&l, c->d_L + (uint64_t)A * c->lplane + (uint64_t)m * c->n_pad + n, sizeof(l),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!((word >> (n & 31)) & 1u)) return CFPQ_ERR_NOT_FOUND;
    if (l == 0xFFFFFFFFu) return CFPQ_ERR_UNSUPPORTED;
    *len = l;
    if (!nodes) return CFPQ_OK;
    if (cap < l) return CFPQ_ERR_BUFFER;
    return lengths_path(c, A, m, n, l, nodes, labels);
}

extern "C" int cfpq_get_all_device(cfpq_ctx *c, cfpq_triple *buf, size_t cap, size_t *count) {
    if (!c || !count) return CFPQ_ERR_INVALID;
    if (!c->solved) return CFPQ_ERR_NOT_SOLVED;
    cudaStream_t s = c->last_stream;
    std::vector<unsigned long long> nt_off;
    int rc = count_all(c, s, nt_off);
    if (rc != CFPQ_OK) return rc;
    const size_t total = (size_t)nt_off[c->n_nt];
    *count = total;
    if (!buf) return CFPQ_OK;
    if (cap < total) return CFPQ_ERR_BUFFER;
    if (total == 0) return CFPQ_OK;
    return emit_all(c, buf, s);
}

extern "C" int cfpq_stats_get(const cfpq_ctx *c, cfpq_stats *out) {
    if (!c || !out) return CFPQ_ERR_INVALID;
    *out = c->stats;
    return CFPQ_OK;
}

extern "C" void cfpq_destroy(cfpq_ctx *c) {
    if (!c) return;
    free_ctx_device(c);
    delete c;
}

extern "C" int cfpq_trim_memory(size_t keep_bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CFPQ_ERR_CUDA;
    }
    cudaMemPool_t pool = cfpq::library_pool(dev);
    if (!pool) return CFPQ_ERR_UNSUPPORTED;
    if (cudaMemPoolTrimTo(pool, keep_bytes) != cudaSuccess) {
        cudaGetLastError();
        return CFPQ_ERR_CUDA;
    }
    return CFPQ_OK;
}
