// Tensor-core (tcgen05) Boolean product path for sm_103a.
//
// One launch computes, for one left-hand side A with productions A -> B_r C_r,
//     P = sum_r T_{B_r} x T_{C_r}      (K-concatenated over the productions)
// on the 5th-generation tensor cores and merges it into T_A: the Boolean product of
// Section 2 (one Boolean matrix product per production, Valiant's |N|^2 reduction) with
// the union T <- T u (T x T) of Algorithm 1 fused into the epilogue.
//
// Exactness: operands are 0 or a positive FP8 E4M3 value (a one at K position q of a byte
// group is the byte 1 << q, 2^-9 .. 2^1, and 0x40 = 2.0 for q = 7; both operands use the
// same values at the same K), products are 0 or at least 2^-18 and are accumulated in F32:
// every term is non-negative, so the sum is non-zero iff some term is, and "accumulator
// != 0" is the Boolean OR of ANDs. (tcgen05 has no 8-bit integer kind on sm_103a.)
//
// Data flow per CTA (one 128 x 256 output tile):
//   warp 0     TMA: bit-packed 128 x 128-bit tile of T_B and 256 x 128-bit tile of T_C^T
//              (the transposed copy, so both operands are K-major) into a packed ring
//   warps 2-17 unpack, in two groups of 8 warps taking alternate K stages (so one group's
//              waits and stores overlap the other's unpacking): 1 bit -> 1 byte. The T_B tile goes straight into tensor memory
//              (tcgen05.st, half a 128-byte K slice per row, lane and warp), the T_C^T tile into
//              shared memory in the 128-byte-swizzled K-major layout. Within each 32-bit
//              word, bit q + 8r becomes byte 4q + r of the word's 32 bytes: the same
//              permutation of K for both operands, so the contraction is unchanged, and
//              each 4 output bytes cost a shift and a mask
//   warp 1     one thread issues tcgen05.mma (M=128, N=256, K=32, A from tensor memory,
//              B from shared memory) into the TMEM accumulator (256 columns)
//   warps 2-17 epilogue: tcgen05.ld, threshold, pack 32 columns per word, OR-merge into
//              T_A, record the new pairs (delta plane, row bitmap), set the change flag
// Every mbarrier wait is bounded (%globaltimer); on expiry the CTA records an error,
// drains what it started and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "cfpq_internal.h"
#include "cfpq_tcgen05.cuh"

namespace cfpq {
namespace tc {

constexpr int BM = 128, BN = 256;
// (the unpacked ring's depth is per kind: Kind<KIND>::UST)
constexpr int B_TILE = BN * 128;      // bytes of one unpacked B stage: 256 rows x 128 bytes
constexpr int UNPACK_GROUPS = 2;     // groups of 8 unpack warps; group g takes the K stages s = g mod 2
constexpr int GROUP_THREADS = 256;   // one group: two warps per SM sub-partition
constexpr int UNPACK_WARPS = 8 * UNPACK_GROUPS;
constexpr uint32_t RASTER_N = 8;      // N tiles per rasterisation band
constexpr int UNPACK_THREADS = 32 * UNPACK_WARPS;
constexpr int THREADS = 64 + UNPACK_THREADS;
constexpr uint32_t ACC_COLS = 256;                 // F32 accumulator, 128 lanes x 256 columns
constexpr uint32_t A_COLS = 32;                    // one stage of A: 128 bytes per lane = 32 columns
// FP4 scale factors (32 columns each, all 2^0) after the accumulator and the UST A stages
template <int UST>
__host__ __device__ constexpr uint32_t sfa_col() { return ACC_COLS + UST * A_COLS; }
template <int UST>
__host__ __device__ constexpr uint32_t sfb_col() { return sfa_col<UST>() + 32; }
constexpr uint32_t TMEM_COLS = 512;                // power of two
static_assert(sfb_col<6>() + 32 <= TMEM_COLS, "tensor memory budget");

// Operand kinds. An unpacked K stage is 128 bytes per row either way (one 128-byte
// swizzle row of a shared-memory tile, 32 tensor-memory columns) and feeds 4 MMAs.
//   KIND 0  E4M3 bytes, kind::f8f6f4 (K = 32 per MMA): a stage is one 128-bit K slice of
//           the bit-packed rows (4 words per row)
//   KIND 1  E2M1 nibbles, kind::mxf4 with unit UE8M0 scale factors (K = 64 per MMA): a
//           stage is two consecutive 128-bit K slices (8 words per row), half the unpacked
//           bytes and half the MMA time per K of KIND 0; dense products, the right operand
//           read as nibbles
//   KIND 2  the same E2M1 MMAs with both operands bit-packed (tile skipping)
template <int KIND>
struct Kind;
template <>
struct Kind<0> {
    static constexpr int KW = 4, PST = 8, SLICES = 1;  // packed words per row and stage, packed ring depth
    static constexpr bool NIBBLE_B = false;            // B arrives bit-packed and is unpacked by the threads
    static constexpr int UST = 5;                      // unpacked ring depth
};
template <>
struct Kind<1> {
    // dense products: B arrives as E2M1 nibbles (T^T kept expanded, k_transpose_e2m1) straight
    // into the MMA's shared-memory layout; a ring slot is the packed A stage plus the B tile,
    // 6 slots (even, so each serves one unpack group)
    // The unpacked A ring has the packed ring's depth (256 + 6 x 32 + 64 tensor-memory columns:
    // all 512), so stage s uses slot s % 6 in both, and one MMA commit per stage frees it in
    // both: the commit follows the unpack's reads of the packed A (the MMAs waited for the
    // unpack), and the loads of stage s + 6, which the unpack waits for, are issued only after it
    static constexpr int KW = 8, PST = 6, SLICES = 2;
    static constexpr bool NIBBLE_B = true;
    static constexpr int UST = 6;
};
template <>
struct Kind<2> {
    // tile skipping: B arrives bit-packed and is unpacked like A (short tiles: a transpose per
    // changed operand and execution writes a quarter of the nibble operand's bytes)
    static constexpr int KW = 8, PST = 5, SLICES = 2;
    static constexpr bool NIBBLE_B = false;
    static constexpr int UST = 5;
};

template <int KIND>
struct __align__(1024) Smem {
    static constexpr int KW = Kind<KIND>::KW, PST = Kind<KIND>::PST, UST = Kind<KIND>::UST;
    static constexpr bool NB = Kind<KIND>::NIBBLE_B;
    uint8_t b_tile[NB ? PST : UST][B_TILE];   // unpacked B stages (nibble B: the ring's B tiles)
    uint32_t a_pack[PST][BM * KW];
    uint32_t b_pack[NB ? 1 : PST][NB ? 4 : BN * KW];  // packed B stages (none with nibble B)
    unsigned long long full_p[PST], empty_p[PST], full_u[UST], empty_u[UST], acc_full, acc_empty;
    unsigned long long mma_done;  // the issuer's last commit: every MMA it issued has completed
    unsigned long long tile_full[2], tile_empty[2];  // tile skipping: claimed tile handed to the consumers
    uint32_t tile_q[2];
    uint32_t tmem_base;
    int err;  // 0, or the wait site that gave up (100: the plan and the bitmaps disagree)
};

template <int KIND>
constexpr size_t smem_bytes() {
    return sizeof(Smem<KIND>) + 1024;
}
static_assert(smem_bytes<0>() <= 227 * 1024 && smem_bytes<1>() <= 227 * 1024 && smem_bytes<2>() <= 227 * 1024,
              "shared memory per CTA");

// Instruction descriptors (both operands K-major, M = 128, N = 256, F32 accumulator):
// kind::f8f6f4 with A = B = E4M3 (bits 4-5: D is F32); kind::mxf4 block-scaled with
// A = B = E2M1 (type 1 in bits 7-9 and 10-12), UE8M0 scale factors (bit 23), scale-factor
// ids 0 (bits 4-5 for B, 29-30 for A).
constexpr uint32_t IDESC_F8 = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) |
                              ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t IDESC_F4 = (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | (1u << 23) |
                              ((uint32_t)(BM >> 4) << 24);

// D[tmem] (+)= A[tmem] x B[smem]^T, E4M3, K = 32
__device__ __forceinline__ void mma_f8_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bd, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}" ::"r"(
            tmem_d),
        "r"(tmem_a), "l"(bd), "r"(IDESC_F8), "r"(accumulate)
        : "memory");
}

// D[tmem] (+)= (A[tmem] x SFA) x (B[smem] x SFB)^T, E2M1, K = 64, one scale factor per 32 K
__device__ __forceinline__ void mma_f4_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bd, uint32_t sfa, uint32_t sfb,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
        " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], [%1], %2, %3, [%4], [%5], p;\n}" ::"r"(
            tmem_d),
        "r"(tmem_a), "l"(bd), "r"(IDESC_F4), "r"(sfa), "r"(sfb), "r"(accumulate)
        : "memory");
}

// The 4 MMAs of one unpacked stage (A at tensor-memory column at, B at shared address bt).
template <int KIND>
__device__ __forceinline__ void mma_stage(uint32_t tmem, uint32_t at, uint32_t bt, bool first) {
    const uint64_t d0 = sdesc(bt);  // the K step kk starts 32 bytes further: + 2 in the address field
#pragma unroll
    for (int kk = 0; kk < 4; kk++) {
        const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
        if constexpr (KIND == 0)
            mma_f8_ts(tmem, at + kk * 8, d0 + (uint64_t)(2 * kk), acc);
        else
            mma_f4_ts(tmem, at + kk * 8, d0 + (uint64_t)(2 * kk), tmem + sfa_col<Kind<KIND>::UST>(),
                      tmem + sfb_col<Kind<KIND>::UST>(), acc);
    }
}

// E4M3: 4 bytes of the unpacked K-row, byte r = bit (q + 8r) of w, as a positive value or 0.
// For q < 7 the bit stays where it is (byte 1 << q: one AND per 4 bytes); bit 7 would be
// the sign, so it moves to bit 6 (0x40 = 2.0).
__device__ __forceinline__ uint32_t spread(uint32_t w, int q) {
    return q < 7 ? (w & (0x01010101u << q)) : ((w >> 1) & 0x40404040u);
}

// E2M1: 8 nibbles of the unpacked K-row, nibble t = bit (4t + s) of w, as a positive value or
// 0. For s < 3 the bit stays where it is (nibble 1 << s = 0.5, 1.0, 2.0: one AND per 8
// nibbles); bit 3 of a nibble would be the sign, so it moves to bit 2 (2.0).
__device__ __forceinline__ uint32_t spread4(uint32_t w, int s) {
    return s < 3 ? (w & (0x11111111u << s)) : ((w >> 1) & 0x44444444u);
}

// Unpacked word u of a stage's K-row (bytes 4u .. 4u+3 of its 128 bytes) from the packed
// words of that row: E4M3 spread(word u / 8, u % 8), E2M1 spread4(word u / 4, u % 4). The
// same permutation of K for both operands, so the contraction is unchanged.
template <int KIND>
__device__ __forceinline__ uint32_t unpacked_word(const uint32_t *w, int u) {
    if constexpr (KIND == 0)
        return spread(w[u >> 3], u & 7);
    else
        return spread4(w[u >> 2], u & 3);
}

// Byte offsets of the 16-byte chunks c = 0..7 of row r in a 128-byte-swizzled K-major tile.
__device__ __forceinline__ void swizzled_row(int r, uint32_t (&off)[8]) {
#pragma unroll
    for (int c = 0; c < 8; c++) off[c] = (uint32_t)r * 128u + ((uint32_t)(c ^ (r & 7)) << 4);
}

// Unpacks one K stage of a row (Kind<KIND>::KW packed words) into its swizzled row of a
// tile (chunk offsets off): chunk c holds the unpacked words 4c .. 4c+3.
template <int KIND>
__device__ __forceinline__ void unpack_row(uint8_t *tile, const uint32_t (&off)[8], const uint32_t *w) {
#pragma unroll
    for (int c = 0; c < 8; c++) {
        uint4 o;
        o.x = unpacked_word<KIND>(w, 4 * c + 0);
        o.y = unpacked_word<KIND>(w, 4 * c + 1);
        o.z = unpacked_word<KIND>(w, 4 * c + 2);
        o.w = unpacked_word<KIND>(w, 4 * c + 3);
        *reinterpret_cast<uint4 *>(tile + off[c]) = o;
    }
}

// Half h of the same K stage of a row (unpacked words 16h .. 16h+15, from the packed words
// w = row + KW h / 2) as 16 tensor-memory columns of one lane: column j of the stage holds
// unpacked word j.
template <int KIND>
__device__ __forceinline__ void unpack_half_row_tmem(uint32_t taddr, const uint32_t *w) {
    uint32_t v[16];
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = unpacked_word<KIND>(w, j);
    tmem_st16(taddr, v);
}

// K slices (bit kb of word w: slice 32 w + kb) that production B x C needs for output tile
// (mt, nt): with tile skipping, those where both operand tiles are non-zero; dense, all.
__device__ __forceinline__ uint32_t live_slices(const QDesc &q, int B, int C, uint32_t mt, uint32_t nt, uint32_t w) {
    if (q.occA) {
        const uint32_t ntiles_m = q.n_pad / BM, ntiles_n = q.n_pad / BN;
        return __ldcg(q.occA + ((uint64_t)B * ntiles_m + mt) * q.SWK + w) &
               __ldcg(q.occB + ((uint64_t)C * ntiles_n + nt) * q.SWK + w);
    }
    const uint32_t left = q.KS - w * 32u;
    return left >= 32u ? 0xFFFFFFFFu : ((1u << left) - 1u);
}

// K stages of a kind in word w of the slice masks: a KIND 1 stage (two slices 2j, 2j + 1,
// bit 2j of the result) is live if either slice is.
template <int KIND>
__device__ __forceinline__ uint32_t live_steps(const QDesc &q, int B, int C, uint32_t mt, uint32_t nt, uint32_t w) {
    const uint32_t x = live_slices(q, B, C, mt, nt, w);
    if constexpr (KIND == 0)
        return x;
    else
        return (x | (x >> 1)) & 0x55555555u;
}

// Output tiles of a product: every N tile of the rows the query computes ([row0, row1)).
__device__ __forceinline__ uint32_t output_tiles(const QDesc &q) { return (q.n_pad / BN) * ((q.row1 - q.row0) / BM); }

// Origin of output tile t of a product (grouped rasterisation: consecutive tiles sweep the M
// tiles of a band of RASTER_N N tiles, so CTAs running at the same time touch about RASTER_N
// right-operand tile columns, which stay in L2).
// The dense E2M1 kernel reads the right operand as nibbles (4x the bytes of a bit-packed band)
// and uses bands of 4 N tiles (measured: 176.6 ms per dense step against 177.5 with 8 and 177.0
// with 2).
__device__ __forceinline__ void tile_origin(const QDesc &q, uint32_t t, uint32_t &m0, uint32_t &n0,
                                            uint32_t raster = RASTER_N) {
    const uint32_t n_tiles = q.n_pad / BN, m_tiles = (q.row1 - q.row0) / BM;
    const uint32_t band = t / (raster * m_tiles);
    const uint32_t first_n = band * raster;
    const uint32_t width = min(raster, n_tiles - first_n);
    const uint32_t local = t - band * raster * m_tiles;
    n0 = (first_n + local % width) * BN;
    m0 = q.row0 + (local / width) * BM;
}

// Tile skipping, one thread per output tile of group g: the tiles with at least one live K
// step (a stage of the product kernel's kind) go to the list as (tile, live K steps); the
// count is the plan slot of this execution.
template <int KIND>
__global__ void __launch_bounds__(256) k_tile_plan(const QDesc *qd, int g, uint2 *list) {
    const QDesc &q = *qd;
    DevState *st = q.st;
    if (st->use_tensor[g] == 0) return;
    const uint32_t tiles = output_tiles(q);
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int r0 = q.gstart[g], r1 = q.gstart[g + 1];
    uint32_t live = 0;
    if (t < tiles) {
        uint32_t m0, n0;
        tile_origin(q, t, m0, n0);
        for (int r = r0; r < r1; r++)
            for (uint32_t w = 0; w < q.SWK; w++)
                live += __popc(live_steps<KIND>(q, q.rules[r].b, q.rules[r].c, m0 / BM, n0 / BN, w));
    }
    const unsigned m = __ballot_sync(0xffffffffu, live != 0u);
    uint32_t base = 0;
    if (lane == 0 && m) base = atomicAdd(&st->plan_count[g][st->iter & 1ull], (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (live) list[base + __popc(m & ((1u << lane) - 1u))] = make_uint2(t, live);
}

// The product of group g over a sequence of output tiles: with list == NULL every tile, CTA b
// taking tiles b, b + grid, ...; with a tile-skipping plan, the live tiles of the list, claimed
// one at a time by the CTA's producer (an atomic on the plan's counter, so CTAs with short tiles
// take more of them) and handed to the MMA and unpack warps through a two-slot ring in shared
// memory. The roles keep one running stage counter across the CTA's tiles; the accumulator is
// handed back by the epilogue (acc_empty) before the next tile's MMAs.
template <int KIND>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_bool_gemm(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmTT, const QDesc *qd,
                   int g, const uint2 *list) {
    constexpr int KW = Kind<KIND>::KW, PST = Kind<KIND>::PST, SLICES = Kind<KIND>::SLICES, UST = Kind<KIND>::UST;
    constexpr bool NB = Kind<KIND>::NIBBLE_B;
    static_assert(!NB || UST == PST, "nibble B: one commit frees both rings' slot");
    static_assert(UNPACK_GROUPS < UST, "a group's ring slot advances by UNPACK_GROUPS with one wrap at most");
    constexpr uint32_t SFA_COL = sfa_col<UST>(), SFB_COL = sfb_col<UST>();
    // N tiles per rasterisation band: 4 for dense nibble products; with a plan list, the plan's own
    // mapping (k_tile_plan numbers tiles with RASTER_N)
    const uint32_t RASTER = (NB && !list) ? 4u : RASTER_N;
    // bytes one K stage brings in: the packed rows of both operands, or (nibble B) the packed A
    // rows and the B tile of E2M1 nibbles (256 rows x 128 bytes)
    constexpr uint32_t STAGE_BYTES = NB ? (uint32_t)BM * KW * 4 + (uint32_t)B_TILE : (uint32_t)(BM + BN) * KW * 4;
    extern __shared__ uint8_t smem_raw[];
    Smem<KIND> &S =
        *reinterpret_cast<Smem<KIND> *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const QDesc &q = *qd;
    DevState *st = q.st;
    if (st->use_tensor[g] == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = q.gstart[g], r1 = q.gstart[g + 1];
    const int A = q.rules[r0].lhs;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->tensor_products, (unsigned long long)(r1 - r0));
    const uint32_t ntile = list ? __ldcg(&st->plan_count[g][st->iter & 1ull]) : output_tiles(q);
    if (blockIdx.x >= ntile) return;  // (uniform over the CTA) no tile for this CTA
    const uint32_t dense_steps = (uint32_t)(r1 - r0) * (q.KS / SLICES);
    volatile int *err = &S.err;

    if (threadIdx.x == 0) {
        for (int i = 0; i < PST; i++) {
            mbar_init(&S.full_p[i], 1);
            // a slot is free once the group has read its packed A (and, nibble B, once the MMAs
            // that read its B tile have completed: one commit)
            mbar_init(&S.empty_p[i], NB ? 1 : GROUP_THREADS);  // nibble B: the MMAs' commit (it follows the unpack's reads)
        }
        for (int i = 0; i < UST; i++) {
            mbar_init(&S.full_u[i], GROUP_THREADS);
            mbar_init(&S.empty_u[i], 1);
        }
        mbar_init(&S.acc_full, 1);
        mbar_init(&S.acc_empty, UNPACK_THREADS);
        mbar_init(&S.mma_done, 1);
        for (int i = 0; i < 2; i++) {
            mbar_init(&S.tile_full[i], 1);
            mbar_init(&S.tile_empty[i], 1 + UNPACK_THREADS);
        }
        S.err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&S.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    constexpr uint32_t kNoTile = 0xFFFFFFFFu;
    unsigned *take = &st->plan_take[g][st->iter & 1ull];
    // ord-th tile of this CTA (the producer claims it; every consumer reads the claim once)
    auto claim_tile = [&](uint32_t ord) -> uint32_t {
        if (!list) {
            const uint64_t i = (uint64_t)blockIdx.x + (uint64_t)ord * gridDim.x;
            return i < ntile ? (uint32_t)i : kNoTile;
        }
        if (!mbar_wait(&S.tile_empty[ord & 1u], ((ord >> 1) & 1u) ^ 1u, err, WAIT_LIMIT_NS, 1)) {
            return kNoTile;
        }
        const uint32_t i = atomicAdd(take, 1u);
        S.tile_q[ord & 1u] = i < ntile ? i : kNoTile;
        mbar_arrive(&S.tile_full[ord & 1u]);
        return i < ntile ? i : kNoTile;
    };
    auto read_tile = [&](uint32_t ord, uint32_t role) -> uint32_t {
        if (!list) {
            const uint64_t i = (uint64_t)blockIdx.x + (uint64_t)ord * gridDim.x;
            return i < ntile ? (uint32_t)i : kNoTile;
        }
        if (!mbar_wait(&S.tile_full[ord & 1u], (ord >> 1) & 1u, err, WAIT_LIMIT_NS, 2)) {
            return kNoTile;
        }
        const uint32_t i = S.tile_q[ord & 1u];
        mbar_arrive(&S.tile_empty[ord & 1u]);
        return i;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: TMA of the bit-packed tiles of each live K step, in the
            // order (production, slice) in which the plan counted them
            uint32_t issued = 0;
            bool stop = false;
            for (uint32_t ord = 0; !stop; ord++) {
                const uint32_t i = claim_tile(ord);
                if (i == kNoTile) break;
                const uint2 e = list ? list[i] : make_uint2(i, dense_steps);
                uint32_t m0, n0;
                tile_origin(q, e.x, m0, n0, RASTER);
                atomicAdd(&st->tc_live_steps, (unsigned long long)e.y * SLICES);  // in 128-bit K slices
                uint32_t done = 0;
                for (int r = r0; r < r1 && !stop; r++) {
                    const int B = q.rules[r].b, C = q.rules[r].c;
                    for (uint32_t w = 0; w < q.SWK && !stop; w++) {
                        uint32_t live = live_steps<KIND>(q, B, C, m0 / BM, n0 / BN, w);
                        while (live && done < e.y) {
                            const uint32_t kb = w * 32u + (uint32_t)(__ffs(live) - 1);
                            live &= live - 1;
                            const uint32_t s = issued;
                            const uint32_t slot = s % PST, ph = (s / PST) & 1u;
                            if (!mbar_wait(&S.empty_p[slot], ph ^ 1u, err, WAIT_LIMIT_NS, 3)) {
                                stop = true;
                                break;
                            }
                            // K slice kb (for KIND 1 the first of the stage's two) starts at word 4 kb
                            // of the packed rows, and at byte 64 kb of the nibble rows
                            mbar_expect_tx(&S.full_p[slot], STAGE_BYTES);
                            tma_load_2d(S.a_pack[slot], &tmT, &S.full_p[slot], (int)(kb * 4u),
                                        (int)((uint32_t)B * q.n_pad + m0));
                            if constexpr (NB)
                                tma_load_2d(S.b_tile[slot], &tmTT, &S.full_p[slot], (int)(kb * 64u),
                                            (int)((uint32_t)C * q.n_pad + n0));
                            else
                                tma_load_2d(S.b_pack[slot], &tmTT, &S.full_p[slot], (int)(kb * 4u),
                                            (int)((uint32_t)C * q.n_pad + n0));
                            issued = s + 1;
                            done++;
                        }
                    }
                }
                if (!stop && done != e.y) {  // the plan and the bitmaps disagree: give up cleanly
                    *err = 100;
                    stop = true;
                }
            }
            if (*err) {
                // drain: the last load issued into each slot must land before the CTA exits
                volatile int drain_err = 0;
                for (uint32_t s = (issued > PST ? issued - PST : 0); s < issued; s++)
                    mbar_wait(&S.full_p[s % PST], (s / PST) & 1u, &drain_err);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            const uint32_t b0 = sa(S.b_tile[0]);
            uint32_t s = 0, tiles_done = 0;
            // running ring positions of stage s: slot = s % UST and its phase, ps = s % PST
            uint32_t slot = 0, ph = 0, ps = 0;
            bool stop = false;
            for (uint32_t ord = 0; !stop; ord++) {
                const uint32_t i = read_tile(ord, 0u);
                if (i == kNoTile) break;
                const uint32_t steps = list ? list[i].y : dense_steps;
                if (tiles_done > 0) {  // the epilogue has read the previous tile's accumulator
                    if (!mbar_wait(&S.acc_empty, (tiles_done - 1) & 1u, err, WAIT_LIMIT_NS, 4)) {
                        break;
                    }
                    tc_fence_after();
                }
                for (uint32_t u = 0; u < steps; u++, s++) {
                    if (!mbar_wait(&S.full_u[slot], ph, err, WAIT_LIMIT_NS, 5)) {
                        stop = true;
                        break;
                    }
                    // nibble B: the stage's B tile has landed. It lands by TMA on full_p[ps] with
                    // the packed A, and the unpack group waited for that phase before its arrivals
                    // on full_u[slot]: passing full_u orders the MMAs after the tile's bytes (a
                    // second wait here, on full_p, cost about 7 % of the dense step)
                    tc_fence_after();
                    const uint32_t at = tmem + ACC_COLS + slot * A_COLS, bt = b0 + (NB ? ps : slot) * B_TILE;
                    mma_stage<KIND>(tmem, at, bt, u == 0);
                    if (NB) mma_commit(&S.empty_p[ps]);  // frees the stage in both rings
                    else mma_commit(&S.empty_u[slot]);
                    if (++slot == (uint32_t)UST) {
                        slot = 0;
                        ph ^= 1u;
                    }
                    if (++ps == (uint32_t)PST) ps = 0;
                }
                mma_commit(&S.acc_full);  // arrives once every MMA issued above has completed
                tiles_done++;
            }
            // On every exit path (a wait that gave up included) the MMAs issued so far must have
            // completed before the tensor memory they write is released: one more commit, and a
            // bounded wait for it that does not stop at the CTA's error flag.
            if (s > 0) {
                mma_commit(&S.mma_done);
                volatile int drain_err = 0;
                mbar_wait(&S.mma_done, 0u, &drain_err);
            }
        }
    } else {
        // ---------------- unpack (8 warps), then the epilogue of each tile
        const int uw = warp - 2;                    // unpack warp 0 .. UNPACK_WARPS-1
        const uint32_t grp = (uint32_t)(uw >> 3);   // K stages s with s % UNPACK_GROUPS == grp
        const int t = (threadIdx.x - 64) & 255;     // the B row of this thread
        const int quad = warp & 3;                  // TMEM lane quadrant this warp may access
        const int half = (uw >> 2) & 1;             // which half of the A slice
        constexpr int CH = (BN / 32) / (UNPACK_WARPS / 4);  // epilogue: 32-column chunks per warp
        const int cq = uw >> 2;                     // ... chunks cq * CH .. cq * CH + CH - 1
        const int arow = quad * 32 + lane;
        const uint32_t a_lane = tmem + ((uint32_t)(quad * 32) << 16) + ACC_COLS + (uint32_t)(16 * half);
        const uint32_t W = q.W;
        const bool inplace = q.schedule == CFPQ_SCHED_INPLACE;
        const uint32_t parity = (uint32_t)(st->iter & 1ull);
        uint32_t *NA = (parity ? q.X0 : q.X1) + (uint64_t)A * q.plane;
        uint32_t *NR = (parity ? q.R0 : q.R1) + (uint64_t)A * W;
        uint32_t *TA = q.T + (uint64_t)A * q.plane;
        uint32_t off[8];
        swizzled_row(t, off);
        if constexpr (KIND != 0) {
            // unit scale factors (UE8M0 127 = 2^0) for every K block of both operands: warps 2-5
            // (one per lane quadrant, all in group 0) write them before their first stage, whose
            // completion the MMA issuer waits for before its first MMA
            if (uw < 4) {
                uint32_t v[32];
#pragma unroll
                for (int j = 0; j < 32; j++) v[j] = 0x7F7F7F7Fu;
                tmem_st32(tmem + ((uint32_t)(quad * 32) << 16) + SFA_COL, v);
                tmem_st32(tmem + ((uint32_t)(quad * 32) << 16) + SFB_COL, v);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
        }
        uint32_t s_end = 0, tiles_done = 0;
        uint32_t sn = grp;                          // this group's next K stage (counted over the CTA's tiles)
        uint32_t us = grp % UST, uph = 0;           // its unpacked ring slot and phase: sn % UST, (sn / UST) & 1
        // this group's stages below limit; false if a wait gave up
        auto unpack_until = [&](uint32_t limit) -> bool {
            for (; sn < limit; sn += UNPACK_GROUPS) {
                const uint32_t ps = sn % PST, pph = (sn / PST) & 1u;
                bool passed = true;
                if constexpr (PST % UNPACK_GROUPS != 0) {
                    // With an odd packed ring the groups take turns on each slot: this group's
                    // waits on full_p[ps] skip every other phase, and a parity wait cannot tell
                    // the phase of stage sn from the one two before it, which is complete while
                    // the other group's stage sn - PST (TMA loads land in any order) may not
                    // have landed yet. So first wait until the other group has consumed stage
                    // sn - PST (phase sn / PST - 1 of empty_p[ps]; the phase before it is this
                    // group's own, already passed): full_p[ps] is then at most one phase behind.
                    if (sn >= (uint32_t)PST) passed = mbar_wait(&S.empty_p[ps], ((sn / PST) - 1u) & 1u, err, WAIT_LIMIT_NS, 9);
                }
                passed = passed && mbar_wait(&S.full_p[ps], pph, err, WAIT_LIMIT_NS, 6);
                // nibble B: stage sn's loads were issued after stage sn - PST's MMAs completed,
                // so the tensor-memory slot (sn % PST) is free once they landed
                if constexpr (!NB) passed = passed && mbar_wait(&S.empty_u[us], uph ^ 1u, err, WAIT_LIMIT_NS, 7);
                // one warp-uniform outcome for the stage: the unpack below uses warp-collective tcgen05.st
                if (!__all_sync(0xffffffffu, passed)) return false;
                tc_fence_after();
                uint32_t pa[KW / 2], pb[KW];  // this lane's half row of A and the thread's row of B
                if constexpr (KIND == 0) {
                    const uint2 x = reinterpret_cast<const uint2 *>(S.a_pack[ps])[2 * arow + half];
                    const uint4 y = reinterpret_cast<const uint4 *>(S.b_pack[ps])[t];
                    pa[0] = x.x, pa[1] = x.y;
                    pb[0] = y.x, pb[1] = y.y, pb[2] = y.z, pb[3] = y.w;
                } else {
                    const uint4 x = reinterpret_cast<const uint4 *>(S.a_pack[ps])[2 * arow + half];
                    pa[0] = x.x, pa[1] = x.y, pa[2] = x.z, pa[3] = x.w;
                    if constexpr (!NB) {
                        const uint4 y0 = reinterpret_cast<const uint4 *>(S.b_pack[ps])[2 * t];
                        const uint4 y1 = reinterpret_cast<const uint4 *>(S.b_pack[ps])[2 * t + 1];
                        pb[0] = y0.x, pb[1] = y0.y, pb[2] = y0.z, pb[3] = y0.w;
                        pb[4] = y1.x, pb[5] = y1.y, pb[6] = y1.z, pb[7] = y1.w;
                    }
                }
                if constexpr (!NB) mbar_arrive(&S.empty_p[ps]);
                unpack_half_row_tmem<KIND>(a_lane + us * A_COLS, pa);
                if constexpr (!NB) {
                    unpack_row<KIND>(S.b_tile[us], off, pb);
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                } else {
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                }
                tc_fence_before();
                mbar_arrive(&S.full_u[us]);
                us += UNPACK_GROUPS;
                if (us >= UST) {
                    us -= UST;
                    uph ^= 1u;
                }
            }
            return true;
        };
        uint32_t ord = 0;  // this CTA's ord-th tile (t is the thread's B row)
        uint32_t i = __shfl_sync(0xffffffffu, read_tile(0, 1u), 0);  // warp-uniform
        uint32_t m0 = 0, n0 = 0;
        if (i != kNoTile) {
            const uint2 e = list ? list[i] : make_uint2(i, dense_steps);
            tile_origin(q, e.x, m0, n0, RASTER);
            s_end = e.y;
        }
        while (i != kNoTile) {
            bool fine = unpack_until(s_end);
            // the next tile's first stages (at most UST: their ring slots are freed by this
            // tile's own MMAs, which wait for nothing else) are unpacked before this tile's
            // epilogue, so that its MMAs can start as soon as the accumulator is handed back
            const uint32_t i2 = __shfl_sync(0xffffffffu, fine ? read_tile(ord + 1, 1u) : kNoTile, 0);  // warp-uniform
            uint32_t m2 = 0, n2 = 0, s_end2 = s_end;
            if (i2 != kNoTile) {
                const uint2 e2 = list ? list[i2] : make_uint2(i2, dense_steps);
                tile_origin(q, e2.x, m2, n2, RASTER);
                s_end2 = s_end + e2.y;
                fine = unpack_until(min(s_end2, s_end + (uint32_t)UST));
            }
            const bool ok =
                __all_sync(0xffffffffu, fine && !*err && mbar_wait(&S.acc_full, tiles_done & 1u, err, WAIT_LIMIT_NS, 8));
            tc_fence_after();
            const uint32_t row = m0 + quad * 32 + lane;
            unsigned cnt = 0;
            uint32_t smask = 0;  // words of this row written in place (one word of the summary of T_A)
#pragma unroll 1
            for (int c = cq * CH; c < (cq + 1) * CH; c++) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c * 32), v);
                uint32_t word = 0;
#pragma unroll
                for (int j = 0; j < 32; j++) word |= (v[j] != 0u ? 1u : 0u) << j;
                if (!ok || *err || row >= q.n || word == 0) continue;
                const uint64_t idx = (uint64_t)row * W + n0 / 32 + c;
                const uint32_t old = __ldcg(TA + idx);
                const uint32_t nw = word & ~old;
                if (nw) {
                    cnt += __popc(nw);
                    if (inplace) TA[idx] = old | nw;
                    NA[idx] = __ldcg(NA + idx) | nw;
                    smask |= 1u << ((n0 / 32u + (uint32_t)c) & 31u);
                }
            }
            if (cnt) {
                atomicOr(&NR[row >> 5], 1u << (row & 31));
                if (inplace) atomicOr(&q.Trow[(uint64_t)A * W + (row >> 5)], 1u << (row & 31));
                if (inplace && q.Tsum) atomicOr(&q.Tsum[((uint64_t)A * q.n_pad + row) * q.SW + (n0 / 32u >> 5)], smask);
            }
            const unsigned any = __ballot_sync(0xffffffffu, cnt != 0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            if (any && lane == 0) {
                atomicAdd(&st->dcount[parity ^ 1u][A], (unsigned long long)cnt);
                atomicAdd(&st->tcount[A], (unsigned long long)cnt);
                atomicAdd(&st->new_bits, (unsigned long long)cnt);
                st->changed = 1u;
                st->dirty[A] = 1u;
                st->odirty[A] = 1u;
            }
            tc_fence_before();
            mbar_arrive(&S.acc_empty);  // the accumulator may be overwritten by the next tile
            tiles_done++;
            if (!ok) break;
            i = i2;
            m0 = m2;
            n0 = n2;
            s_end = s_end2;
            ord++;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && S.err) {
        atomicExch(&st->error, kErrDevice);
        if (atomicCAS(&st->tc_diag[0], 0u, (unsigned)S.err) == 0u) {
            st->tc_diag[1] = blockIdx.x + 1u;
            st->tc_diag[2] = (unsigned)g;
            st->tc_diag[3] = (unsigned)st->iter;
            st->tc_diag[4] = ntile;
            st->tc_diag[5] = list ? __ldcg(take) : 0u;
        }
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Transpose of a 32 x 32 bit block held one row per lane (bit j of lane i = element (i, j)):
// afterwards lane j holds column j (bit i = element (i, j)). Five butterfly steps; in step s the
// lanes l and l ^ s exchange the off-diagonal s x s blocks of each 2s x 2s block.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; k++) {
        const int sh = 16 >> k;
        const uint32_t m = masks[k];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sh);
        x = (lane & sh) ? ((x & ~m) | ((y >> sh) & m)) : ((x & m) | ((y << sh) & ~m));
    }
    return x;
}

// Bit-matrix transpose of plane a: TT[a] = T[a]^T. One CTA: 256 rows x 8 words (256 x 256 bits);
// warp w reads rows 32 w .. 32 w + 31 (one row per lane, its 8 words as two 16-byte loads),
// transposes the 8 blocks of 32 x 32 bits in registers and stages them for row-wise stores.
// gate >= 0 (AUTO path): only if the per-iteration choice assigned this refresh to group gate.
__global__ void __launch_bounds__(256) k_transpose(const QDesc *qd, int a, int gate) {
    __shared__ uint32_t out[256][9];
    const QDesc &q = *qd;
    if (gate >= 0 && q.st->tt_now[a] != (unsigned)gate + 1u) return;
    const uint32_t W = q.W;
    const uint32_t r0 = blockIdx.y * 256, wc0 = blockIdx.x * 8;
    const uint32_t *src = q.T + (uint64_t)a * q.plane;
    uint32_t *dst = q.TT + (uint64_t)a * q.plane;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // W is a multiple of 8 and wc0 of 8: the row's 8 words are 32-byte aligned
    const uint4 *row = reinterpret_cast<const uint4 *>(src + (uint64_t)(r0 + t) * W + wc0);
    const uint4 lo = __ldcg(row), hi = __ldcg(row + 1);
    const uint32_t in[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (int c = 0; c < 8; c++) out[c * 32 + lane][warp] = transpose32(in[c], lane);
    __syncthreads();
    // output row wc0 * 32 + t: words r0 / 32 .. r0 / 32 + 7 (32-byte aligned: r0 is a multiple of 256)
    uint4 *drow = reinterpret_cast<uint4 *>(dst + (uint64_t)(wc0 * 32 + t) * W + r0 / 32);
    drow[0] = make_uint4(out[t][0], out[t][1], out[t][2], out[t][3]);
    drow[1] = make_uint4(out[t][4], out[t][5], out[t][6], out[t][7]);
}

// T_a^T as E2M1 nibbles, the right operand of the E2M1 product (TMA loads its K stages straight
// into the MMA's 128-byte-swizzled shared-memory layout). Row r of TTn[a] is n_pad / 2 bytes;
// the 128 bytes of K stage st (K = 256 st .. 256 st + 255) are the 32 unpacked words
// u = 0 .. 31, word u = spread4(word 8 st + u / 4 of row r of T_a^T, u % 4): the K permutation
// with which the product unpacks its left operand, so both operands agree. One CTA per 256
// rows x 256 columns of T_a, as k_transpose; each thread writes the 128 bytes of one stage of
// one output row.
__global__ void __launch_bounds__(256) k_transpose_e2m1(const QDesc *qd, int a, int gate, uint8_t *ttn) {
    __shared__ uint32_t out[256][9];
    const QDesc &q = *qd;
    if (gate >= 0 && q.st->tt_now[a] != (unsigned)gate + 1u) return;
    const uint32_t W = q.W;
    const uint32_t r0 = blockIdx.y * 256, wc0 = blockIdx.x * 8;
    const uint32_t *src = q.T + (uint64_t)a * q.plane;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint4 *row = reinterpret_cast<const uint4 *>(src + (uint64_t)(r0 + t) * W + wc0);
    const uint4 lo = __ldcg(row), hi = __ldcg(row + 1);
    const uint32_t in[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (int c = 0; c < 8; c++) out[c * 32 + lane][warp] = transpose32(in[c], lane);
    __syncthreads();
    // output rows wc0 * 32 + 0 .. 255, K stage r0 / 256: each row's 8 packed words become its 128
    // bytes (chunk k = the 4 unpacked words of packed word k); 8 consecutive threads write one
    // row, so a warp's store covers 4 whole 128-byte lines
    const uint64_t rb = (uint64_t)q.n_pad / 2u;  // bytes per nibble row
    uint8_t *base = ttn + ((uint64_t)a * q.n_pad + wc0 * 32) * rb + (r0 / 256u) * 128u;
#pragma unroll
    for (int it = 0; it < 8; it++) {
        const int c = it * 256 + t, r = c >> 3, k = c & 7;
        const uint32_t v = out[r][k];
        reinterpret_cast<uint4 *>(base + (uint64_t)r * rb)[k] = make_uint4(spread4(v, 0), spread4(v, 1), spread4(v, 2), spread4(v, 3));
    }
}

// Tile occupancy of T_a for tile skipping (one CTA per 256 rows x 256 columns, as k_transpose):
// the CTA's 2 x 2 blocks of 128 rows x 128 columns give two (m-tile, K slice) bits of occA[a]
// per m-tile and, ORed over the columns, the two (n-tile, K slice) bits of occB[a] (T_a^T's
// tile of 256 rows x 128 columns is T_a's 128 rows x 256 columns). Each bit belongs to exactly
// one CTA, which writes it whether set or clear (no clearing pass) and adds the bits it flips
// to the per-(non-terminal, K slice) counts of non-zero tiles that the automatic path's cost
// model reads (occCA: m-tiles, occCB: n-tiles). Runs only if the plan of this execution asks
// for a (occ_now) and some group takes the tensor product now, or the cost model asked for
// the counts (occ_probe).
__device__ __forceinline__ void count_flips(uint32_t *cnt, uint32_t old_word, uint32_t new_word, uint32_t sh) {
#pragma unroll
    for (uint32_t kk = 0; kk < 2; kk++) {
        const uint32_t ob = (old_word >> (sh + kk)) & 1u, nb = (new_word >> (sh + kk)) & 1u;
        if (ob != nb) atomicAdd(cnt + kk, nb ? 1u : 0xFFFFFFFFu);
    }
}

__global__ void __launch_bounds__(256) k_occupancy(const QDesc *qd, int a) {
    const QDesc &q = *qd;
    const DevState *st = q.st;
    if (!st->occ_now[a]) return;
    unsigned any_tc = st->occ_probe;
    for (int g = 0; g < q.n_groups; g++) any_tc |= st->use_tensor[g];
    if (!any_tc) return;
    __shared__ uint32_t mask;
    if (threadIdx.x == 0) mask = 0u;
    __syncthreads();
    const uint32_t r0 = blockIdx.y * 256u, wc0 = blockIdx.x * 8u;
    const uint32_t *src = q.T + (uint64_t)a * q.plane;
    uint32_t m = 0;
    for (int idx = threadIdx.x; idx < 2048; idx += 256) {
        const uint32_t row = (uint32_t)idx >> 3, w = (uint32_t)idx & 7u;
        if (__ldcg(src + (uint64_t)(r0 + row) * q.W + wc0 + w)) m |= 1u << ((row >> 7) * 2u + (w >> 2));
    }
    m = __reduce_or_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicOr(&mask, m);
    __syncthreads();
    if (threadIdx.x != 0) return;
    const uint32_t M = mask;
    const uint32_t ntiles_m = q.n_pad / BM, ntiles_n = q.n_pad / BN;
    const uint32_t ks = wc0 / 4u;  // first of the two K slices of the columns (even)
    for (uint32_t h = 0; h < 2; h++) {
        uint32_t *word = q.occA + ((uint64_t)a * ntiles_m + r0 / BM + h) * q.SWK + ks / 32u;
        const uint32_t bits = ((M >> (2u * h)) & 3u) << (ks & 31u);
        const uint32_t old = atomicAnd(word, ~(3u << (ks & 31u)));
        if (bits) atomicOr(word, bits);
        if (q.occCA) count_flips(q.occCA + (uint64_t)a * q.KS + ks, old, bits, ks & 31u);
    }
    const uint32_t ksr = r0 / 128u;  // the two K slices of the rows (even), as T_a^T columns
    const uint32_t rb = ((M | (M >> 1)) & 1u) | (((M >> 2) | (M >> 3)) & 1u) << 1;
    uint32_t *wordB = q.occB + ((uint64_t)a * ntiles_n + wc0 / 8u) * q.SWK + ksr / 32u;
    const uint32_t oldB = atomicAnd(wordB, ~(3u << (ksr & 31u)));
    if (rb) atomicOr(wordB, rb << (ksr & 31u));
    if (q.occCB) count_flips(q.occCB + (uint64_t)a * q.KS + ksr, oldB, rb << (ksr & 31u), ksr & 31u);
    if (blockIdx.x == 0 && blockIdx.y == 0 && q.occKnown) q.occKnown[a] = 1u;
}

// Profile mode, useful work of one tensor product T_B x T_C: sum over k of the ones in
// column k of T_B times the ones in row k of T_C (the multiply-adds with both operands 1).
// Column counts: one thread per column of a 256-column band, over 256 rows per block.
__global__ void __launch_bounds__(256) k_colcount(const QDesc *qd, int b, uint32_t *colcnt) {
    const QDesc &q = *qd;
    const uint32_t w = blockIdx.x * 8u + (threadIdx.x >> 5), bit = threadIdx.x & 31u;
    const uint32_t r0 = blockIdx.y * 256u;
    const uint32_t *src = q.T + (uint64_t)b * q.plane;
    uint32_t cnt = 0;
    for (uint32_t i = r0; i < r0 + 256u && i < q.n; i++) cnt += (__ldcg(src + (uint64_t)i * q.W + w) >> bit) & 1u;
    if (cnt) atomicAdd(&colcnt[w * 32u + bit], cnt);
}

// Row counts of T_C (one warp per row), then the dot product with the column counts.
__global__ void __launch_bounds__(256) k_useful_dot(const QDesc *qd, int c, int g, const uint32_t *colcnt) {
    const QDesc &q = *qd;
    if (q.st->use_tensor[g] == 0) return;  // this product ran on the gather path
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= q.n) return;
    const uint32_t *row = q.T + (uint64_t)c * q.plane + warp * q.W;
    uint32_t cnt = 0;
    for (uint32_t w = lane; w < q.W; w += 32) cnt += __popc(__ldcg(row + w));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0 && cnt) atomicAdd(&q.st->useful_macs, (unsigned long long)cnt * colcnt[warp]);
}

}  // namespace tc

// ------------------------------------------------------------------------------------ host

// Profile mode: adds the useful multiply-adds of group g's tensor products (at the operands'
// current contents, which are what the products read) to the device state.
int enqueue_useful_work(cfpq_ctx *c, int g, cudaStream_t s) {
    for (int r = c->gstart[g]; r < c->gstart[g + 1]; r++) {
        if (cudaMemsetAsync(c->d_colcnt, 0, sizeof(uint32_t) * c->n_pad, s) != cudaSuccess) return CFPQ_ERR_CUDA;
        tc::k_colcount<<<dim3(c->W / 8, c->n_pad / 256), 256, 0, s>>>(c->d_q, c->rules[r].b, c->d_colcnt);
        tc::k_useful_dot<<<(uint32_t)(((uint64_t)c->n * 32 + 255) / 256), 256, 0, s>>>(c->d_q, c->rules[r].c, g,
                                                                                       c->d_colcnt);
    }
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

static int g_tc_available = -1;

bool tensor_path_available() {
    if (g_tc_available < 0) {
        int dev = 0;
        cudaDeviceProp p;
        g_tc_available = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&p, dev) == cudaSuccess)
            g_tc_available = (p.major == 10 && p.minor == 3) ? 1 : 0;
        cudaGetLastError();
    }
    return g_tc_available == 1;
}

struct TensorWork {
    CUtensorMap tmT[3], tmTT[3];  // per operand kind: boxes of Kind<KIND>::KW words (tmTT[1]: nibbles)
    bool attr_set;
};

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// The E2M1 right operand: nibble rows of n_pad / 2 bytes, boxes of one K stage (128 bytes) x
// box_rows rows, 128-byte swizzle (the MMA's K-major shared-memory layout).
static bool encode_nibble_map(CUtensorMap *m, uint8_t *base, const cfpq_ctx *c, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)c->n_pad / 2, (cuuint64_t)c->n_nt * c->n_pad};
    const cuuint64_t strides[1] = {(cuuint64_t)c->n_pad / 2};
    const cuuint32_t box[2] = {128u, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

static bool encode_map(CUtensorMap *m, uint32_t *base, const cfpq_ctx *c, uint32_t box_words, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {c->W, (cuuint64_t)c->n_nt * c->n_pad};
    const cuuint64_t strides[1] = {(cuuint64_t)c->W * 4};
    const cuuint32_t box[2] = {(cuuint32_t)box_words, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// Dense E2M1 products read the right operand as nibbles (KIND 1); tile skipping (a plan list)
// and E4M3 products read it bit-packed.
static bool uses_nibble_operand(const cfpq_ctx *c) {
    return c->tensor_kind != CFPQ_TENSOR_FP8 && c->dense_tensor;
}

static int tensor_setup(cfpq_ctx *c) {
    if (c->h_tc_work) return CFPQ_OK;  // once per context
    if (!c->d_TT) return CFPQ_ERR_UNSUPPORTED;
    if (uses_nibble_operand(c) && !c->d_TTn) {
        // the dense E2M1 products' right operand, made at the first tensor set-up of the
        // context (contexts that never take a tensor product do not hold it)
        void *p = nullptr;
        const size_t bytes = (size_t)c->n_nt * c->n_pad * (c->n_pad / 2);
        const cudaError_t e = ctx_alloc(c, &p, bytes, c->stream);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CFPQ_ERR_NOMEM : CFPQ_ERR_CUDA;
        c->d_TTn = static_cast<uint8_t *>(p);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return CFPQ_ERR_CUDA;  // used on any stream
    }
    TensorWork *w = new TensorWork();
    memset(w, 0, sizeof(*w));
    if (!encode_map(&w->tmT[0], c->d_T, c, tc::Kind<0>::KW, tc::BM) ||
        !encode_map(&w->tmTT[0], c->d_TT, c, tc::Kind<0>::KW, tc::BN) ||
        !encode_map(&w->tmT[1], c->d_T, c, tc::Kind<1>::KW, tc::BM) ||
        (c->d_TTn && !encode_nibble_map(&w->tmTT[1], c->d_TTn, c, tc::BN)) ||
        !encode_map(&w->tmT[2], c->d_T, c, tc::Kind<2>::KW, tc::BM) ||
        !encode_map(&w->tmTT[2], c->d_TT, c, tc::Kind<2>::KW, tc::BN)) {
        delete w;
        return CFPQ_ERR_CUDA;
    }
    if (cudaFuncSetAttribute(tc::k_tc_bool_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc::smem_bytes<0>()) != cudaSuccess ||
        cudaFuncSetAttribute(tc::k_tc_bool_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc::smem_bytes<1>()) != cudaSuccess ||
        cudaFuncSetAttribute(tc::k_tc_bool_gemm<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc::smem_bytes<2>()) != cudaSuccess) {
        delete w;
        return CFPQ_ERR_CUDA;
    }
    c->h_tc_work = w;
    c->d_tc_work = nullptr;
    return CFPQ_OK;
}

void tensor_release(cfpq_ctx *c) {
    delete static_cast<TensorWork *>(c->h_tc_work);
    c->h_tc_work = nullptr;
}

// The right operand of a tensor product: T_a^T as nibbles for dense E2M1 products, bit-packed
// otherwise.
static void launch_transpose(cfpq_ctx *c, int a, cudaStream_t s, int64_t *launches, int gate = -1) {
    const dim3 grid(c->W / 8, c->n_pad / 256);
    if (uses_nibble_operand(c))
        tc::k_transpose_e2m1<<<grid, 256, 0, s>>>(c->d_q, a, gate, c->d_TTn);
    else
        tc::k_transpose<<<grid, 256, 0, s>>>(c->d_q, a, gate);
    (*launches)++;
}

// AUTO path: transposes of the group's right operands, each run only if this iteration's
// choice (k_choose) assigned its refresh to group g.
int enqueue_tensor_transposes_gated(cfpq_ctx *c, int g, cudaStream_t s) {
    const int rc = tensor_setup(c);
    if (rc != CFPQ_OK) return rc;
    std::vector<char> done(c->n_nt, 0);
    int64_t ignored = 0;
    for (int r = c->gstart[g]; r < c->gstart[g + 1]; r++) {
        const int C = c->rules[r].c;
        if (done[C]) continue;
        done[C] = 1;
        launch_transpose(c, C, s, &ignored, g);
    }
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

int tensor_prepare(cfpq_ctx *c) { return tensor_setup(c); }

// Tile occupancy of every operand of a tensor-capable group (tile skipping); each launch
// returns at once unless this execution's plan asks for it and a tensor product runs now.
int enqueue_tensor_occupancy(cfpq_ctx *c, cudaStream_t s) {
    if (!c->d_occA) return CFPQ_OK;
    std::vector<char> need(c->n_nt, 0);
    for (int g = 0; g < c->n_groups; g++)
        for (int r = c->gstart[g]; r < c->gstart[g + 1]; r++) need[c->rules[r].b] = need[c->rules[r].c] = 1;
    const dim3 grid(c->W / 8, c->n_pad / 256);
    for (int a = 0; a < c->n_nt; a++)
        if (need[a]) {
            tc::k_occupancy<<<grid, 256, 0, s>>>(c->d_q, a);
            c->iter_launches++;
        }
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

// T^T (bit-packed) of every non-terminal that a production derives (the worklist's hand-over).
int enqueue_transpose_bits(cfpq_ctx *c, int a, cudaStream_t s) {
    tc::k_transpose<<<dim3(c->W / 8, c->n_pad / 256), 256, 0, s>>>(c->d_q, a, -1);
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

int enqueue_all_transposes(cfpq_ctx *c, cudaStream_t s) {
    for (int a = 0; a < c->n_nt; a++)
        if (c->nt_dynamic[a] && enqueue_transpose_bits(c, a, s) != CFPQ_OK) return CFPQ_ERR_CUDA;
    return CFPQ_OK;
}

// After the matrix initialisation: transposes of every right operand of a tensor group.
int enqueue_tensor_seed_transposes(cfpq_ctx *c, cudaStream_t s, int64_t *launches) {
    int rc = tensor_setup(c);
    if (rc != CFPQ_OK) return rc;
    std::vector<char> done(c->n_nt, 0);
    for (int g = 0; g < c->n_groups; g++) {
        if (!c->group_tensor[g]) continue;
        for (int r = c->gstart[g]; r < c->gstart[g + 1]; r++) {
            const int C = c->rules[r].c;
            if (done[C]) continue;
            done[C] = 1;
            launch_transpose(c, C, s, launches);
        }
    }
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

// Refreshes the transposes of the group's right operands that may have changed.
int enqueue_tensor_transposes(cfpq_ctx *c, int g, cudaStream_t s) {
    const int rc = tensor_setup(c);
    if (rc != CFPQ_OK) return rc;
    std::vector<char> done(c->n_nt, 0);
    for (int r = c->gstart[g]; r < c->gstart[g + 1]; r++) {
        const int C = c->rules[r].c;
        if (done[C] || !c->nt_dynamic[C]) continue;
        done[C] = 1;
        launch_transpose(c, C, s, &c->iter_launches);
    }
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

// The tensor-core product of group g (after enqueue_tensor_transposes), with the operand
// kind of the context (c->tensor_kind: 1 E4M3, 2 E2M1).
template <int KIND>
static void launch_group(cfpq_ctx *c, TensorWork *w, int g, cudaStream_t s, uint32_t tiles, uint32_t grid) {
    if (c->d_tile_list) {
        // tile skipping: list the live output tiles, then one CTA per SM over the list
        tc::k_tile_plan<KIND><<<(tiles + 255) / 256, 256, 0, s>>>(c->d_q, g, reinterpret_cast<uint2 *>(c->d_tile_list));
        tc::k_tc_bool_gemm<KIND><<<grid, tc::THREADS, tc::smem_bytes<KIND>(), s>>>(
            w->tmT[KIND], w->tmTT[KIND], c->d_q, g, reinterpret_cast<const uint2 *>(c->d_tile_list));
        c->iter_launches += 2;
    } else {
        tc::k_tc_bool_gemm<KIND><<<grid, tc::THREADS, tc::smem_bytes<KIND>(), s>>>(w->tmT[KIND], w->tmTT[KIND],
                                                                                 c->d_q, g, nullptr);
        c->iter_launches++;
    }
}

int enqueue_tensor_group(cfpq_ctx *c, int g, cudaStream_t s) {
    const int rc = tensor_setup(c);
    if (rc != CFPQ_OK) return rc;
    TensorWork *w = static_cast<TensorWork *>(c->h_tc_work);
    const uint32_t tiles = (c->n_pad / tc::BN) * ((c->row1 - c->row0) / tc::BM);  // the row block's tiles
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t grid = std::min<uint32_t>(tiles, (uint32_t)std::max(1, sms));
    if (c->tensor_kind == CFPQ_TENSOR_FP8)
        launch_group<0>(c, w, g, s, tiles, grid);
    else if (uses_nibble_operand(c))
        launch_group<1>(c, w, g, s, tiles, grid);
    else
        launch_group<2>(c, w, g, s, tiles, grid);
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

}  // namespace cfpq
