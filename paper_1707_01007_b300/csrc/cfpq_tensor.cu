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

namespace cfpq {
namespace tc {

constexpr int BM = 128, BN = 256;
constexpr int KW = 4;                 // 32-bit words of K per stage
constexpr int BK = 32 * KW;           // 128 K elements per stage
constexpr int PST = 8, UST = 5;       // packed / unpacked ring depths
constexpr int A_PACK = BM * KW * 4, B_PACK = BN * KW * 4;  // bytes of one packed stage
constexpr int B_TILE = BN * BK;       // bytes of one unpacked B stage (FP8)
constexpr int UNPACK_GROUPS = 2;     // groups of 8 unpack warps; group g takes the K stages s = g mod 2
constexpr int GROUP_THREADS = 256;   // one group: two warps per SM sub-partition
constexpr int UNPACK_WARPS = 8 * UNPACK_GROUPS;
static_assert(UNPACK_GROUPS < UST, "a group's ring slot advances by UNPACK_GROUPS with one wrap at most");
constexpr uint32_t RASTER_N = 8;      // N tiles per rasterisation band
constexpr int UNPACK_THREADS = 32 * UNPACK_WARPS;
constexpr int THREADS = 64 + UNPACK_THREADS;
constexpr uint32_t ACC_COLS = 256;                 // F32 accumulator, 128 lanes x 256 columns
constexpr uint32_t A_COLS = BK / 4;                // one stage of A: 128 FP8 per lane = 32 columns
constexpr uint32_t TMEM_COLS = 512;                // accumulator + UST stages of A, power of two
static_assert(ACC_COLS + UST * A_COLS <= TMEM_COLS, "tensor memory budget");
constexpr unsigned long long WAIT_LIMIT_NS = 2ull * 1000 * 1000 * 1000;  // 2 s per wait

struct __align__(1024) Smem {
    uint8_t b_tile[UST][B_TILE];
    uint32_t a_pack[PST][BM * KW];
    uint32_t b_pack[PST][BN * KW];
    unsigned long long full_p[PST], empty_p[PST], full_u[UST], empty_u[UST], acc_full, acc_empty;
    unsigned long long mma_done;  // the issuer's last commit: every MMA it issued has completed
    unsigned long long tile_full[2], tile_empty[2];  // tile skipping: claimed tile handed to the consumers
    uint32_t tile_q[2];
    uint32_t tmem_base;
    int err;
};

constexpr size_t SMEM_BYTES = sizeof(Smem) + 1024;

__device__ __forceinline__ uint32_t sa(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(unsigned long long *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(sa(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and the CTA's error flag set) if the phase did not complete in time
// or another role of the CTA already gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, uint32_t parity, volatile int *err) {
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try(b, parity)) return true;
        if (*err) return false;
        if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) {
            *err = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, unsigned long long *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(sa(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading-dimension byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride-dimension byte offset
    d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::f8f6f4, A = B = E4M3, D = F32, both K-major, M x N.
constexpr uint32_t IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

// D[tmem] (+)= A[tmem] x B[smem]^T
__device__ __forceinline__ void mma_f8_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bd, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}" ::"r"(
            tmem_d),
        "r"(tmem_a), "l"(bd), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

// 4 bytes of the unpacked K-row: byte r = bit (q + 8r) of w, as a positive FP8 E4M3 value or
// 0. For q < 7 the bit stays where it is (byte 1 << q: one AND per 4 bytes); bit 7 would be
// the sign, so it moves to bit 6 (0x40 = 2.0).
__device__ __forceinline__ uint32_t spread(uint32_t w, int q) {
    return q < 7 ? (w & (0x01010101u << q)) : ((w >> 1) & 0x40404040u);
}

// Byte offsets of the 16-byte chunks c = 0..7 of row r in a 128-byte-swizzled K-major tile.
__device__ __forceinline__ void swizzled_row(int r, uint32_t (&off)[8]) {
#pragma unroll
    for (int c = 0; c < 8; c++) off[c] = (uint32_t)r * 128u + ((uint32_t)(c ^ (r & 7)) << 4);
}

// Unpacks one 128-bit K slice of a row into its swizzled row of a tile (chunk offsets off).
__device__ __forceinline__ void unpack_row(uint8_t *tile, const uint32_t (&off)[8], uint4 p) {
    const uint32_t w[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
    for (int wi = 0; wi < 4; wi++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            uint4 o;
            o.x = spread(w[wi], 4 * h + 0);
            o.y = spread(w[wi], 4 * h + 1);
            o.z = spread(w[wi], 4 * h + 2);
            o.w = spread(w[wi], 4 * h + 3);
            *reinterpret_cast<uint4 *>(tile + off[wi * 2 + h]) = o;
        }
}

// Half (64 bytes, words 2h and 2h+1) of the same 128-byte K slice as unpack_row, as 16 TMEM
// columns of one lane: column j of the slice holds logical bytes 4j .. 4j+3, i.e.
// spread(word j/8, j%8); this half is columns 16h .. 16h+15.
__device__ __forceinline__ void unpack_half_row_tmem(uint32_t taddr, uint2 p) {
    uint32_t v[16];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        v[j] = spread(p.x, j);
        v[8 + j] = spread(p.y, j);
    }
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

// Origin of output tile t of a product (grouped rasterisation: consecutive tiles sweep the M
// tiles of a band of RASTER_N N tiles, so CTAs running at the same time touch about RASTER_N
// right-operand tile columns, which stay in L2).
__device__ __forceinline__ void tile_origin(const QDesc &q, uint32_t t, uint32_t &m0, uint32_t &n0) {
    const uint32_t n_tiles = q.n_pad / BN, m_tiles = q.n_pad / BM;
    const uint32_t band = t / (RASTER_N * m_tiles);
    const uint32_t first_n = band * RASTER_N;
    const uint32_t width = min((uint32_t)RASTER_N, n_tiles - first_n);
    const uint32_t local = t - band * RASTER_N * m_tiles;
    n0 = (first_n + local % width) * BN;
    m0 = (local / width) * BM;
}

// Tile skipping, one thread per output tile of group g: the tiles with at least one live K
// step go to the list as (tile, live K steps); the count is the plan slot of this execution.
__global__ void __launch_bounds__(256) k_tile_plan(const QDesc *qd, int g, uint2 *list) {
    const QDesc &q = *qd;
    DevState *st = q.st;
    if (st->use_tensor[g] == 0) return;
    const uint32_t tiles = (q.n_pad / BN) * (q.n_pad / BM);
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int r0 = q.gstart[g], r1 = q.gstart[g + 1];
    uint32_t live = 0;
    if (t < tiles) {
        uint32_t m0, n0;
        tile_origin(q, t, m0, n0);
        for (int r = r0; r < r1; r++)
            for (uint32_t w = 0; w < q.SWK; w++)
                live += __popc(live_slices(q, q.rules[r].b, q.rules[r].c, m0 / BM, n0 / BN, w));
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
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_bool_gemm(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmTT, const QDesc *qd,
                   int g, const uint2 *list) {
    extern __shared__ uint8_t smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const QDesc &q = *qd;
    DevState *st = q.st;
    if (st->use_tensor[g] == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = q.gstart[g], r1 = q.gstart[g + 1];
    const int A = q.rules[r0].lhs;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->tensor_products, (unsigned long long)(r1 - r0));
    const uint32_t ntile = list ? __ldcg(&st->plan_count[g][st->iter & 1ull]) : (q.n_pad / BN) * (q.n_pad / BM);
    if (blockIdx.x >= ntile) return;  // (uniform over the CTA) no tile for this CTA
    const uint32_t dense_steps = (uint32_t)(r1 - r0) * q.KS;
    volatile int *err = &S.err;

    if (threadIdx.x == 0) {
        for (int i = 0; i < PST; i++) {
            mbar_init(&S.full_p[i], 1);
            mbar_init(&S.empty_p[i], GROUP_THREADS);
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
        if (!mbar_wait(&S.tile_empty[ord & 1u], ((ord >> 1) & 1u) ^ 1u, err)) return kNoTile;
        const uint32_t i = atomicAdd(take, 1u);
        S.tile_q[ord & 1u] = i < ntile ? i : kNoTile;
        mbar_arrive(&S.tile_full[ord & 1u]);
        return i < ntile ? i : kNoTile;
    };
    auto read_tile = [&](uint32_t ord) -> uint32_t {
        if (!list) {
            const uint64_t i = (uint64_t)blockIdx.x + (uint64_t)ord * gridDim.x;
            return i < ntile ? (uint32_t)i : kNoTile;
        }
        if (!mbar_wait(&S.tile_full[ord & 1u], (ord >> 1) & 1u, err)) return kNoTile;
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
                tile_origin(q, e.x, m0, n0);
                atomicAdd(&st->tc_live_steps, (unsigned long long)e.y);
                uint32_t done = 0;
                for (int r = r0; r < r1 && !stop; r++) {
                    const int B = q.rules[r].b, C = q.rules[r].c;
                    for (uint32_t w = 0; w < q.SWK && !stop; w++) {
                        uint32_t live = live_slices(q, B, C, m0 / BM, n0 / BN, w);
                        while (live && done < e.y) {
                            const uint32_t kb = w * 32u + (uint32_t)(__ffs(live) - 1);
                            live &= live - 1;
                            const uint32_t s = issued;
                            const uint32_t slot = s % PST, ph = (s / PST) & 1u;
                            if (!mbar_wait(&S.empty_p[slot], ph ^ 1u, err)) {
                                stop = true;
                                break;
                            }
                            mbar_expect_tx(&S.full_p[slot], A_PACK + B_PACK);
                            tma_load_2d(S.a_pack[slot], &tmT, &S.full_p[slot], (int)(kb * KW),
                                        (int)((uint32_t)B * q.n_pad + m0));
                            tma_load_2d(S.b_pack[slot], &tmTT, &S.full_p[slot], (int)(kb * KW),
                                        (int)((uint32_t)C * q.n_pad + n0));
                            issued = s + 1;
                            done++;
                        }
                    }
                }
                if (!stop && done != e.y) {  // the plan and the bitmaps disagree: give up cleanly
                    *err = 1;
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
            bool stop = false;
            for (uint32_t ord = 0; !stop; ord++) {
                const uint32_t i = read_tile(ord);
                if (i == kNoTile) break;
                const uint32_t steps = list ? list[i].y : dense_steps;
                if (tiles_done > 0) {  // the epilogue has read the previous tile's accumulator
                    if (!mbar_wait(&S.acc_empty, (tiles_done - 1) & 1u, err)) break;
                    tc_fence_after();
                }
                for (uint32_t u = 0; u < steps; u++, s++) {
                    const uint32_t slot = s % UST, ph = (s / UST) & 1u;
                    if (!mbar_wait(&S.full_u[slot], ph, err)) {
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t at = tmem + ACC_COLS + slot * A_COLS, bt = b0 + slot * B_TILE;
#pragma unroll
                    for (int kk = 0; kk < BK / 32; kk++)
                        mma_f8_ts(tmem, at + kk * 8, sdesc(bt + kk * 32), (u > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(&S.empty_u[slot]);
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
        uint32_t s_end = 0, tiles_done = 0;
        uint32_t sn = grp;                          // this group's next K stage (counted over the CTA's tiles)
        uint32_t us = grp % UST, uph = 0;           // its unpacked ring slot and phase: sn % UST, (sn / UST) & 1
        // this group's stages below limit; false if a wait gave up
        auto unpack_until = [&](uint32_t limit) -> bool {
            for (; sn < limit; sn += UNPACK_GROUPS) {
                const uint32_t ps = sn % PST, pph = (sn / PST) & 1u;
                if (!mbar_wait(&S.full_p[ps], pph, err)) return false;
                if (!mbar_wait(&S.empty_u[us], uph ^ 1u, err)) return false;
                tc_fence_after();
                const uint2 pa = reinterpret_cast<const uint2 *>(S.a_pack[ps])[2 * arow + half];
                const uint4 pb = reinterpret_cast<const uint4 *>(S.b_pack[ps])[t];
                mbar_arrive(&S.empty_p[ps]);
                unpack_half_row_tmem(a_lane + us * A_COLS, pa);
                unpack_row(S.b_tile[us], off, pb);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
        uint32_t i = read_tile(0);
        uint32_t m0 = 0, n0 = 0;
        if (i != kNoTile) {
            const uint2 e = list ? list[i] : make_uint2(i, dense_steps);
            tile_origin(q, e.x, m0, n0);
            s_end = e.y;
        }
        while (i != kNoTile) {
            bool fine = unpack_until(s_end);
            // the next tile's first stages (at most UST: their ring slots are freed by this
            // tile's own MMAs, which wait for nothing else) are unpacked before this tile's
            // epilogue, so that its MMAs can start as soon as the accumulator is handed back
            const uint32_t i2 = fine ? read_tile(ord + 1) : kNoTile;
            uint32_t m2 = 0, n2 = 0, s_end2 = s_end;
            if (i2 != kNoTile) {
                const uint2 e2 = list ? list[i2] : make_uint2(i2, dense_steps);
                tile_origin(q, e2.x, m2, n2);
                s_end2 = s_end + e2.y;
                fine = unpack_until(min(s_end2, s_end + (uint32_t)UST));
            }
            const bool ok = fine && !*err && mbar_wait(&S.acc_full, tiles_done & 1u, err);
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
    if (threadIdx.x == 0 && S.err) atomicExch(&st->error, 3u);
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

// Tile occupancy of T_a for tile skipping (one CTA per 256 rows x 256 columns, as k_transpose):
// the CTA's 2 x 2 blocks of 128 rows x 128 columns give two (m-tile, K slice) bits of occA[a]
// per m-tile and, ORed over the columns, the two (n-tile, K slice) bits of occB[a] (T_a^T's
// tile of 256 rows x 128 columns is T_a's 128 rows x 256 columns). Each bit belongs to exactly
// one CTA, which writes it whether set or clear (no clearing pass). Runs only if the plan of
// this execution asks for a (occ_now) and some group takes the tensor product now.
__global__ void __launch_bounds__(256) k_occupancy(const QDesc *qd, int a) {
    const QDesc &q = *qd;
    const DevState *st = q.st;
    if (!st->occ_now[a]) return;
    unsigned any_tc = 0u;
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
        atomicAnd(word, ~(3u << (ks & 31u)));
        if (bits) atomicOr(word, bits);
    }
    const uint32_t ksr = r0 / 128u;  // the two K slices of the rows (even), as T_a^T columns
    const uint32_t rb = ((M | (M >> 1)) & 1u) | (((M >> 2) | (M >> 3)) & 1u) << 1;
    uint32_t *wordB = q.occB + ((uint64_t)a * ntiles_n + wc0 / 8u) * q.SWK + ksr / 32u;
    atomicAnd(wordB, ~(3u << (ksr & 31u)));
    if (rb) atomicOr(wordB, rb << (ksr & 31u));
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
    CUtensorMap tmT, tmTT;
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

static bool encode_map(CUtensorMap *m, uint32_t *base, const cfpq_ctx *c, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {c->W, (cuuint64_t)c->n_nt * c->n_pad};
    const cuuint64_t strides[1] = {(cuuint64_t)c->W * 4};
    const cuuint32_t box[2] = {(cuuint32_t)tc::KW, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

static int tensor_setup(cfpq_ctx *c) {
    if (c->d_tc_work) return CFPQ_OK;
    if (!c->d_TT) return CFPQ_ERR_UNSUPPORTED;
    TensorWork *w = new TensorWork();
    memset(w, 0, sizeof(*w));
    if (!encode_map(&w->tmT, c->d_T, c, tc::BM) || !encode_map(&w->tmTT, c->d_TT, c, tc::BN)) {
        delete w;
        return CFPQ_ERR_CUDA;
    }
    if (cudaFuncSetAttribute(tc::k_tc_bool_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM_BYTES) !=
        cudaSuccess) {
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

static void launch_transpose(cfpq_ctx *c, int a, cudaStream_t s, int64_t *launches, int gate = -1) {
    const dim3 grid(c->W / 8, c->n_pad / 256);
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

// T^T of every non-terminal that a production derives (the worklist's hand-over).
int enqueue_all_transposes(cfpq_ctx *c, cudaStream_t s) {
    int64_t ignored = 0;
    for (int a = 0; a < c->n_nt; a++)
        if (c->nt_dynamic[a]) launch_transpose(c, a, s, &ignored);
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
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

// The tensor-core product of group g (after enqueue_tensor_transposes).
int enqueue_tensor_group(cfpq_ctx *c, int g, cudaStream_t s) {
    const int rc = tensor_setup(c);
    if (rc != CFPQ_OK) return rc;
    TensorWork *w = static_cast<TensorWork *>(c->h_tc_work);
    const uint32_t tiles = (c->n_pad / tc::BN) * (c->n_pad / tc::BM);
    if (c->d_tile_list) {
        // tile skipping: list the live output tiles, then one CTA per SM over the list
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        tc::k_tile_plan<<<(tiles + 255) / 256, 256, 0, s>>>(c->d_q, g, reinterpret_cast<uint2 *>(c->d_tile_list));
        const uint32_t grid = std::min<uint32_t>(tiles, (uint32_t)std::max(1, sms));
        tc::k_tc_bool_gemm<<<grid, tc::THREADS, tc::SMEM_BYTES, s>>>(w->tmT, w->tmTT, c->d_q, g,
                                                                    reinterpret_cast<const uint2 *>(c->d_tile_list));
        c->iter_launches += 2;
    } else {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const uint32_t grid = std::min<uint32_t>(tiles, (uint32_t)std::max(1, sms));
        tc::k_tc_bool_gemm<<<grid, tc::THREADS, tc::SMEM_BYTES, s>>>(w->tmT, w->tmTT, c->d_q, g, nullptr);
        c->iter_launches++;
    }
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

}  // namespace cfpq
