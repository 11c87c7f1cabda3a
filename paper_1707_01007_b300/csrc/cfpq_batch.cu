// Batched closure: many independent queries advanced together by one persistent
// (cooperative) launch. Each round performs one execution of Algorithm 1's loop body
// (Section 4.2) for every query that has not converged; a query whose round added no
// pair is retired while the others continue (per-query convergence). All queries share
// the grid: work items (query, production group, row, column chunk) are spread over
// all warps, so small and large queries overlap on the device.
//
// Every wait in this file (the grid barrier) is bounded by a %globaltimer deadline;
// on expiry the kernel records an error and returns.
//
// The launch configuration (persistent grid size, gather tile width per size class, and
// the schedule of CFPQ_SCHED_AUTO queries) comes from a process-wide table that the
// autotuner at the end of this file fills by timing candidate configurations on the
// caller's own batch.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "cfpq_batch.h"
#include "cfpq_internal.h"

namespace cfpq {

constexpr unsigned long long kBarrierTimeoutNs = 20ull * 1000 * 1000 * 1000;    // 20 s
constexpr unsigned long long kLaunchLimitNs = 600ull * 1000 * 1000 * 1000;     // 10 min per launch

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier on one counter: block 0 adds 2^31 - (G - 1), every other block adds
// 1, so the counter's top bit flips exactly when all G blocks have arrived (no reset, no
// separate generation word). Arrival is a release (fence + atomic), polling an acquire
// load. The wait is bounded; returns false (the same value in every thread of the block)
// once any block has recorded an error.
__device__ bool grid_barrier(BatchCtl *ctl) {
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned nb = blockIdx.x == 0 ? (0x80000000u - (gridDim.x - 1u)) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(&ctl->bar_count, nb);
        unsigned ok = 1;
        const unsigned long long t0 = globaltimer_ns();
        for (;;) {
            const unsigned cur = ld_acquire_u32(&ctl->bar_count);
            if ((old ^ cur) & 0x80000000u) break;
            if (ld_acquire_u32(&ctl->error)) { ok = 0; break; }
            if (globaltimer_ns() - t0 > kBarrierTimeoutNs) {
                atomicExch(&ctl->error, 1u);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_ok = ok && ld_acquire_u32(&ctl->error) == 0u;
    }
    __syncthreads();
    return s_ok != 0u;
}

// index of the slot containing item x in offsets[0..n] (offsets[0] = 0, increasing)
__device__ __forceinline__ int find_slot(const unsigned long long *off, int n, unsigned long long x) {
    int lo = 0, hi = n;  // off[lo] <= x < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldcg(off + mid) <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// The same search in a block's shared copy of the offsets.
__device__ __forceinline__ int find_slot_shared(const unsigned long long *off, int n, unsigned long long x) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Rounds with at most this many queries take part read the round's tables (item offsets,
// row offsets, query ids) from a shared-memory copy in every block.
constexpr int kSlotCache = 1024;

// Rebuilds the per-round tables over the queries that take part in round `round`: not
// converged and still within their own round budget (one block of <= 1024 threads).
__device__ void build_tables(BatchCtl *ctl, const BatchQuery *bq, int round) {
    __shared__ unsigned long long sp[1024], sr[1024];
    __shared__ int sa[1024];
    const int k = ctl->k;
    const int per = (k + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(k, lo + per);
    unsigned long long p = 0, r = 0;
    int a = 0;
    for (int j = lo; j < hi; j++)
        if (__ldcg(ctl->active + j) && round < bq[j].max_rounds) {
            a++;
            p += bq[j].prod_items;
            r += bq[j].row_items;
        }
    sp[threadIdx.x] = p;
    sr[threadIdx.x] = r;
    sa[threadIdx.x] = a;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const unsigned long long vp = threadIdx.x >= (unsigned)off ? sp[threadIdx.x - off] : 0ull;
        const unsigned long long vr = threadIdx.x >= (unsigned)off ? sr[threadIdx.x - off] : 0ull;
        const int va = threadIdx.x >= (unsigned)off ? sa[threadIdx.x - off] : 0;
        __syncthreads();
        sp[threadIdx.x] += vp;
        sr[threadIdx.x] += vr;
        sa[threadIdx.x] += va;
        __syncthreads();
    }
    unsigned long long P = sp[threadIdx.x] - p, R = sr[threadIdx.x] - r;
    int A = sa[threadIdx.x] - a;
    for (int j = lo; j < hi; j++)
        if (__ldcg(ctl->active + j) && round < bq[j].max_rounds) {
            ctl->act[A] = j;
            ctl->prod_off[A] = P;
            ctl->row_off[A] = R;
            A++;
            P += bq[j].prod_items;
            R += bq[j].row_items;
        }
    if (threadIdx.x == blockDim.x - 1) {
        ctl->n_active = (unsigned)A;
        ctl->list_len = 0;  // every reader of the previous list has passed a barrier since
        ctl->prod_off[A] = P;
        ctl->row_off[A] = R;
    }
    __syncthreads();
}

constexpr unsigned long long kClrChunk = 2048;   // uint4 per clear item (32 KB)
constexpr unsigned long long kSeedChunk = 256;   // edges or eps pairs per seed item

// query j with off(j) <= x < off(j+1) for a start-phase prefix field (clr_off or seed_off)
template <unsigned long long BatchQuery::*OFF>
__device__ __forceinline__ int find_query(const BatchQuery *bq, int k, unsigned long long x) {
    int lo = 0, hi = k;  // invariant: bq[lo].*OFF <= x, and x < bq[hi].*OFF when hi < k
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bq[mid].*OFF <= x) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void zero_span(uint4 *p, unsigned long long lo, unsigned long long hi, int lane) {
    for (unsigned long long w = lo + lane; w < hi; w += 32) p[w] = make_uint4(0, 0, 0, 0);
}

// Product item: query j (24 bits), group g (8), row i (20), column chunk ch (12).
__device__ __forceinline__ unsigned long long pack_item(int j, int g, uint32_t i, uint32_t ch) {
    return ((unsigned long long)j << 40) | ((unsigned long long)g << 32) | ((unsigned long long)i << 12) | ch;
}
__device__ __forceinline__ void unpack_item(unsigned long long v, int *j, int *g, uint32_t *i, uint32_t *ch) {
    *j = (int)(v >> 40);
    *g = (int)((v >> 32) & 0xFFu);
    *i = (uint32_t)((v >> 12) & 0xFFFFFu);
    *ch = (uint32_t)(v & 0xFFFu);
}


// 4 blocks of 256 per SM (registers capped at 64; a few spill): the phases are latency-bound and
// gain more from resident warps than they lose to the spills (measured 4.7 -> 4.1 ms on 256 queries)
__global__ void __launch_bounds__(256, 4) k_batch(BatchCtl *ctl, const BatchQuery *bq) {
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gwarp = gtid >> 5, gwarps = gthreads >> 5;
    const int lane = threadIdx.x & 31;
    const int k = ctl->k;
    if (gtid == 0) ctl->start_ns = globaltimer_ns();

    // 1) queries starting in this launch: clear their matrices (chunks over all such
    //    queries) and reset their state
    for (unsigned long long it = gwarp; it < ctl->clr_total; it += gwarps) {
        const int j = find_query<&BatchQuery::clr_off>(bq, k, it);
        const BatchQuery &b = bq[j];
        const unsigned long long c = it - b.clr_off;
        const unsigned long long ca = (b.clr_a_n + kClrChunk - 1) / kClrChunk;
        if (c < ca) zero_span(b.clr_a, c * kClrChunk, min(b.clr_a_n, (c + 1) * kClrChunk), lane);
        else zero_span(b.clr_b, (c - ca) * kClrChunk, min(b.clr_b_n, (c - ca + 1) * kClrChunk), lane);
    }
    for (int j = (int)gwarp; j < k; j += (int)gwarps) {  // a warp zeroes a new query's state
        if (!bq[j].init) continue;
        const QDesc &q = bq[j].q;
        DevState *st = q.st;
        unsigned long long *w = reinterpret_cast<unsigned long long *>(st);
        for (int i = lane; i < (int)(sizeof(DevState) / 8); i += 32) w[i] = 0ull;
        __syncwarp();
        if (lane == 0) st->max_iter = bq[j].max_iter;
        for (int a = lane; a < q.n_nt; a += 32) st->dirty[a] = 1u;
    }
    if (!grid_barrier(ctl)) return;
    // 2) matrix initialisation of the new queries (chunks of edges, then of eps pairs); the new
    // pairs are counted per non-terminal in the warp's shared table and added to the query's
    // counts once per chunk (not one global atomic per pair on the same few addresses)
    __shared__ unsigned s_seed_cnt[256 / 32][kMaxNT];
    unsigned *wcnt = s_seed_cnt[threadIdx.x >> 5];
    for (unsigned long long it = gwarp; it < ctl->seed_total; it += gwarps) {
        const int j = find_query<&BatchQuery::seed_off>(bq, k, it);
        const QDesc &q = bq[j].q;
        const unsigned long long items = q.n_edges + (unsigned long long)q.n_eps * q.n;
        const unsigned long long lo = (it - bq[j].seed_off) * kSeedChunk;
        const unsigned long long hi = min(items, lo + kSeedChunk);
        for (int a = lane; a < q.n_nt; a += 32) wcnt[a] = 0u;
        __syncwarp();
        unsigned long long cnt = 0;
        for (unsigned long long e = lo + lane; e < hi; e += 32) {
            if (e < q.n_edges) {
                const cfpq_edge ed = q.edges[e];
                for (int u = 0; u < q.n_unary; u++)
                    if (q.unary[u].y == ed.label) seed_pair(q, q.unary[u].x, ed.src, ed.dst, &cnt, wcnt);
            } else {
                const unsigned long long t = e - q.n_edges;
                const uint32_t m = (uint32_t)(t % q.n);
                seed_pair(q, q.eps[t / q.n], m, m, &cnt, wcnt);
            }
        }
        __syncwarp();
        for (int a = lane; a < q.n_nt; a += 32)
            if (wcnt[a]) {
                atomicAdd(&q.st->dcount[0][a], (unsigned long long)wcnt[a]);
                atomicAdd(&q.st->tcount[a], (unsigned long long)wcnt[a]);
            }
        const unsigned wsum = __reduce_add_sync(0xffffffffu, (unsigned)cnt);
        if (lane == 0 && wsum) atomicAdd(&q.st->seed_bits, (unsigned long long)wsum);
        __syncwarp();  // the table is reset by the next item only after every lane has read it
    }
    if (!grid_barrier(ctl)) return;
    if (blockIdx.x == 0) build_tables(ctl, bq, 0);
    if (!grid_barrier(ctl)) return;
    // phase clock (block 0, thread 0): time from the previous barrier to this one
    unsigned long long t_prev = 0;
    auto mark = [&](int phase, int round) {
        if (gtid == 0) {
            const unsigned long long t = globaltimer_ns();
            const unsigned long long d = t - (phase == 0 ? ctl->start_ns : t_prev);
            ctl->phase_ns[phase] += d;
            if (phase == 2 && round < kProfRounds) ctl->round_product_ns[round] = d;
            t_prev = t;
        }
    };
    mark(0, 0);

    __shared__ unsigned long long s_poff[kSlotCache + 1], s_roff[kSlotCache + 1];
    __shared__ int s_act[kSlotCache];
    for (int round = 0; round < ctl->max_rounds; round++) {
        const int na = min((int)ld_u32(&ctl->n_active), k);
        if (na <= 0) break;
        if (gtid == 0) ctl->rounds++;
        // the round's tables (built by block 0 before the last barrier), once per block: each
        // lane's search for its item's query then costs no global round trips
        const bool cached = na <= kSlotCache;
        if (cached) {
            for (int i = threadIdx.x; i <= na; i += blockDim.x) {
                s_poff[i] = __ldcg(ctl->prod_off + i);
                s_roff[i] = __ldcg(ctl->row_off + i);
                if (i < na) s_act[i] = __ldcg(ctl->act + i);
            }
            __syncthreads();
        }
        // query and offset within it of item `it` of a table (prod or row offsets)
        auto slot_of = [&](bool rows_table, unsigned long long it, int &jj, unsigned long long &loc) {
            if (cached) {
                const unsigned long long *off = rows_table ? s_roff : s_poff;
                const int sl = find_slot_shared(off, na, it);
                jj = s_act[sl];
                loc = it - off[sl];
            } else {
                const unsigned long long *off = rows_table ? ctl->row_off : ctl->prod_off;
                const int sl = find_slot(off, na, it);
                jj = __ldcg(ctl->act + sl);
                loc = it - __ldcg(off + sl);
            }
        };
        // 3a) candidate rows, one lane per item (query, group, row word): the rows of the
        //     word that have a left delta row or (where the right operand has a delta) a
        //     non-empty left row become one product item per column chunk; the warp reserves
        //     its lanes' items with one atomic and each lane writes its own
        const unsigned long long np = cached ? s_poff[na] : __ldcg(ctl->prod_off + na);
        for (unsigned long long it0 = gwarp * 32ull; it0 < np; it0 += gwarps * 32ull) {
            const unsigned long long it = it0 + (unsigned)lane;
            uint32_t cand = 0, wq = 0, nch = 0;
            int j = 0, g = 0;
            if (it < np) {
                unsigned long long loc = 0;
                slot_of(false, it, j, loc);
                if (j >= 0 && j < k) {
                    const BatchQuery &b = bq[j];
                    const QDesc &q = b.q;
                    const uint32_t rw = (q.n + 31u) / 32u;
                    const unsigned long long g64 = loc / rw;
                    wq = (uint32_t)(loc % rw);
                    if (g64 < (unsigned long long)q.n_groups) {
                        g = (int)g64;
                        nch = b.nch;
                        const uint32_t parity = (uint32_t)(ld_u64(&q.st->iter) & 1ull);
                        const uint32_t *DR = parity ? q.R1 : q.R0;
                        // a production's three loads are independent: issued together
#pragma unroll 4
                        for (int ri = q.gstart[g]; ri < q.gstart[g + 1]; ri++) {
                            const int B = q.rules[ri].b, C = q.rules[ri].c;
                            const uint32_t d = __ldcg(DR + (uint64_t)B * q.W + wq);
                            const unsigned long long dc = ld_u64(&q.st->dcount[parity][C]);
                            const uint32_t t = __ldcg(q.Trow + (uint64_t)B * q.W + wq);
                            cand |= d | (dc != 0ull ? t : 0u);
                        }
                        cand &= rows_in_word(q.n, wq);
                    }
                }
            }
            const uint32_t cnt = (uint32_t)__popc(cand) * nch;
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const uint32_t wtotal = __shfl_sync(0xffffffffu, incl, 31);
            if (wtotal == 0) continue;
            unsigned long long base = 0;
            if (lane == 31) base = atomicAdd(&ctl->list_len, (unsigned long long)wtotal);
            base = __shfl_sync(0xffffffffu, base, 31);
            if (base + wtotal > ctl->list_cap) {  // cannot happen: the capacity covers every row
                if (lane == 0) atomicExch(&ctl->error, 3u);
                continue;
            }
            unsigned long long pos = base + incl - cnt;
            while (cand) {
                const uint32_t i = wq * 32u + (uint32_t)(__ffs(cand) - 1);
                cand &= cand - 1;
                for (uint32_t ch = 0; ch < nch; ch++) ctl->list[pos++] = pack_item(j, g, i, ch);
            }
        }
        // the plane this round's products write (N) is the one the previous round read (its
        // D): its row bitmap is zeroed (one lane per (query, non-terminal, row word)). Its rows
        // are not: the products write every chunk of a row they touch whole (gather_row_chunk
        // with WRITE_CHUNK), a row is read again only where its bit is set, and a set bit means
        // every chunk of the row was written in this round.
        const unsigned long long nr = cached ? s_roff[na] : __ldcg(ctl->row_off + na);
        for (unsigned long long it = gwarp * 32ull + (unsigned)lane; it < nr; it += gwarps * 32ull) {
            int j = 0;
            unsigned long long loc = 0;
            slot_of(true, it, j, loc);
            if (j >= 0 && j < k && loc < bq[j].row_items) {
                const QDesc &q = bq[j].q;
                const uint32_t rw = (q.n + 31u) / 32u;
                const uint32_t prev = (uint32_t)((ld_u64(&q.st->iter) + 1ull) & 1ull);
                uint32_t *bm = (prev ? q.R1 : q.R0) + (uint64_t)(loc / rw) * q.W + (uint32_t)(loc % rw);
                if (__ldcg(bm)) *bm = 0u;
            }
        }
        if (!grid_barrier(ctl)) return;
        mark(1, round);
        // 3b) products of the listed items (one warp per row chunk)
        const unsigned long long nl = min(__ldcg(&ctl->list_len), ctl->list_cap);
        for (unsigned long long it = gwarp; it < nl; it += gwarps) {
            int j, g;
            uint32_t i, ch;
            unpack_item(__ldcg(ctl->list + it), &j, &g, &i, &ch);
            if (j >= k) continue;
            const BatchQuery &b = bq[j];
            if (g >= b.q.n_groups || i >= b.q.n || ch >= b.nch) continue;
            const uint32_t parity = (uint32_t)(ld_u64(&b.q.st->iter) & 1ull);
            switch (b.cpl) {
                case 1: gather_row_chunk<1, true>(b.q, g, i, ch, lane, parity); break;
                case 2: gather_row_chunk<2, true>(b.q, g, i, ch, lane, parity); break;
                case 4: gather_row_chunk<4, true>(b.q, g, i, ch, lane, parity); break;
                default: gather_row_chunk<8, true>(b.q, g, i, ch, lane, parity); break;
            }
        }
        if (!grid_barrier(ctl)) return;
        mark(2, round);
        // 4) Jacobi queries: T |= N over the rows N touched (one lane per (query, non-terminal,
        //    row word) finds them and sets the row bitmap of T; the warp merges them together)
        if (ctl->any_jacobi) {
            const unsigned long long nr = cached ? s_roff[na] : __ldcg(ctl->row_off + na);
            for (unsigned long long it0 = gwarp * 32ull; it0 < nr; it0 += gwarps * 32ull) {
                const unsigned long long it = it0 + (unsigned)lane;
                uint32_t rows = 0, wq = 0, W = 0;
                uint32_t *tp = nullptr;
                const uint32_t *np_ = nullptr;
                if (it < nr) {
                    int j = 0;
                    unsigned long long loc = 0;
                    slot_of(true, it, j, loc);
                    if (j >= 0 && j < k && loc < bq[j].row_items && bq[j].q.schedule == CFPQ_SCHED_JACOBI) {
                        const QDesc &q = bq[j].q;
                        const uint32_t rw = (q.n + 31u) / 32u;
                        const int a = (int)(loc / rw);
                        wq = (uint32_t)(loc % rw);
                        W = q.W;
                        const uint32_t parity = (uint32_t)(ld_u64(&q.st->iter) & 1ull);
                        rows = __ldcg((parity ? q.R0 : q.R1) + (uint64_t)a * q.W + wq) & rows_in_word(q.n, wq);
                        tp = q.T + (uint64_t)a * q.plane;
                        np_ = (parity ? q.X0 : q.X1) + (uint64_t)a * q.plane;
                        if (rows) atomicOr(&q.Trow[(uint64_t)a * q.W + wq], rows);
                    }
                }
                unsigned todo = __ballot_sync(0xffffffffu, rows != 0);
                while (todo) {
                    const int src = __ffs(todo) - 1;
                    todo &= todo - 1;
                    uint32_t r = __shfl_sync(0xffffffffu, rows, src);
                    const uint32_t sw = __shfl_sync(0xffffffffu, W, src), swq = __shfl_sync(0xffffffffu, wq, src);
                    uint32_t *st_ = reinterpret_cast<uint32_t *>(
                        __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(tp), src));
                    const uint32_t *sn = reinterpret_cast<const uint32_t *>(
                        __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(np_), src));
                    while (r) {
                        const uint64_t i = swq * 32u + (uint32_t)(__ffs(r) - 1);
                        r &= r - 1;
                        for (uint32_t w = lane; w < sw; w += 32) {
                            const uint32_t nw = __ldcg(sn + i * sw + w);
                            if (nw) st_[i * sw + w] = __ldcg(st_ + i * sw + w) | nw;
                        }
                    }
                }
            }
            if (!grid_barrier(ctl)) return;
            mark(3, round);
        }
        // 6) per-query end of iteration; a converged query is retired
        for (int s = blockIdx.x; s < na; s += gridDim.x) {
            const int j = __ldcg(ctl->act + s);
            if (j < 0 || j >= k) continue;  // uniform across the block
            const unsigned cont = tail_query(bq[j].q, threadIdx.x, blockDim.x, false);
            if (threadIdx.x == 0) {
                bq[j].q.st->gather_products += (unsigned long long)bq[j].q.n_rules;
                if (!cont) ctl->active[j] = 0;
            }
            __syncthreads();
        }
        // every tail must be done (it reads act[] and writes active[]) before the tables change
        if (!grid_barrier(ctl)) return;
        mark(4, round);
        if (blockIdx.x == 0) {
            build_tables(ctl, bq, round + 1);
            if (threadIdx.x == 0 && ctl->limit_ns && globaltimer_ns() - ctl->start_ns > ctl->limit_ns)
                atomicExch(&ctl->error, 2u);
            __syncthreads();
        }
        if (!grid_barrier(ctl)) return;
        mark(5, round);
    }
}

int batch_launch(BatchCtl *d_ctl, const BatchQuery *d_bq, cudaStream_t s, int blocks_per_sm, int *grid_out) {
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CFPQ_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return CFPQ_ERR_UNSUPPORTED;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, 256, 0) != cudaSuccess || per_sm < 1)
        return CFPQ_ERR_CUDA;
    // a cooperative grid must be co-resident: never more blocks per SM than occupancy allows
    const int bps = blocks_per_sm > 0 ? std::min(blocks_per_sm, per_sm) : std::min(per_sm, 8);
    const int grid = sms * bps;
    void *args[] = {(void *)&d_ctl, (void *)&d_bq};
    if (cudaLaunchCooperativeKernel((const void *)k_batch, dim3(grid), dim3(256), args, 0, s) != cudaSuccess)
        return CFPQ_ERR_CUDA;
    if (grid_out) *grid_out = grid;
    return CFPQ_OK;
}

// ------------------------------------------------------------------------------------ tuning

int batch_size_class(uint32_t W) {
    int c = 0;
    while (c < CFPQ_TUNE_CLASSES - 1 && (1u << c) < W) c++;
    return c;
}

static std::mutex g_tune_mu;
static cfpq_batch_tuning g_tune = [] {
    cfpq_batch_tuning t;
    cfpq_batch_tuning_default(&t);
    return t;
}();

void batch_tuning_snapshot(cfpq_batch_tuning *t) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    *t = g_tune;
}

static bool tuning_valid(const cfpq_batch_tuning &t) {
    if (t.blocks_per_sm < 0 || t.blocks_per_sm > 8) return false;
    for (int c = 0; c < CFPQ_TUNE_CLASSES; c++) {
        const int v = t.cpl[c];
        if (v != 0 && v != 1 && v != 2 && v != 4 && v != 8) return false;
        if (t.schedule[c] != CFPQ_SCHED_INPLACE && t.schedule[c] != CFPQ_SCHED_JACOBI) return false;
        if (t.product[c] != CFPQ_BATCH_GROUPED && t.product[c] != CFPQ_BATCH_ALONE) return false;
    }
    return true;
}

void fill_batch_query(const cfpq_ctx *c, BatchQuery *b, int init, const cfpq_batch_tuning &t) {
    memset(b, 0, sizeof(*b));
    b->q = c->hq;
    b->q.allow_switch = 0;  // the grouped launch runs every query by the matrix loop
    b->q.occA = b->q.occB = nullptr;  // gather products only: no tile occupancy, no length summaries
    b->q.Tsum = b->q.TTsum = nullptr;
    const int cls = batch_size_class(c->W);
    int cpl = 1;
    uint32_t nch = gather_chunks(c->W, &cpl);
    if (t.cpl[cls] > 0) {
        cpl = t.cpl[cls];
        nch = (c->W + 32u * (uint32_t)cpl - 1) / (32u * (uint32_t)cpl);
    }
    b->cpl = cpl;
    b->nch = nch;
    if (c->schedule_req == CFPQ_SCHED_AUTO) b->q.schedule = t.schedule[cls];
    const unsigned long long rw = (c->n + 31u) / 32u;  // row words: 32 rows per work item
    b->prod_items = (unsigned long long)c->n_groups * rw;
    b->row_slots = (unsigned long long)c->n_groups * c->n * nch;
    b->row_items = (unsigned long long)c->n_nt * rw;
    b->init = init;
    b->max_iter = c->max_iter;
    // [T, X1 end) and [R0, Trow end) are contiguous in the query's arena (parts are
    // 256-byte aligned and padded, so both spans are whole uint4s)
    const size_t planes = (size_t)c->n_nt * c->plane * 4;
    const size_t rowsz = ((size_t)c->n_nt * c->W * 4 + 255) / 256 * 256;
    b->clr_a = reinterpret_cast<uint4 *>(c->d_T);
    b->clr_a_n = 3 * planes / 16;
    b->clr_b = reinterpret_cast<uint4 *>(c->d_R0);
    b->clr_b_n = ((size_t)(reinterpret_cast<char *>(c->d_Trow) - reinterpret_cast<char *>(c->d_R0)) + rowsz) / 16;
    b->max_rounds = 1 << 30;
}

int batch_buffers_alloc(BatchBuffers *b, int k) {
    memset(b, 0, sizeof(*b));
    b->k = k;
    if (cudaMalloc(&b->ctl, sizeof(BatchCtl)) != cudaSuccess ||
        cudaMalloc(&b->bq, sizeof(BatchQuery) * k) != cudaSuccess ||
        cudaMalloc(&b->active, sizeof(int) * k) != cudaSuccess ||
        cudaMalloc(&b->act, sizeof(int) * k) != cudaSuccess ||
        cudaMalloc(&b->prod_off, sizeof(unsigned long long) * (k + 1)) != cudaSuccess ||
        cudaMalloc(&b->row_off, sizeof(unsigned long long) * (k + 1)) != cudaSuccess ||
        cudaMalloc(&b->states, sizeof(DevState) * k) != cudaSuccess) {
        cudaGetLastError();
        batch_buffers_free(b);
        return CFPQ_ERR_NOMEM;
    }
    return CFPQ_OK;
}

int batch_buffers_upload(BatchBuffers *b, BatchQuery *hb, const int *active, int k, int max_rounds,
                         bool any_jacobi, cudaStream_t s, unsigned long long limit_ns) {
    BatchCtl ctl;
    memset(&ctl, 0, sizeof(ctl));
    unsigned long long clr = 0, seed = 0;
    for (int j = 0; j < k; j++) {
        hb[j].clr_off = clr;
        hb[j].seed_off = seed;
        if (!hb[j].init) continue;
        clr += (hb[j].clr_a_n + kClrChunk - 1) / kClrChunk + (hb[j].clr_b_n + kClrChunk - 1) / kClrChunk;
        const unsigned long long items = hb[j].q.n_edges + (unsigned long long)hb[j].q.n_eps * hb[j].q.n;
        seed += (items + kSeedChunk - 1) / kSeedChunk;
    }
    ctl.clr_total = clr;
    ctl.seed_total = seed;
    unsigned long long slots = 0;
    for (int j = 0; j < k; j++) slots += hb[j].row_slots;
    if (slots > b->list_cap) {
        const unsigned long long cap = std::max(slots, 2 * b->list_cap);
        if (b->list) cudaFree(b->list);
        b->list = nullptr;
        b->list_cap = 0;
        if (cudaMalloc(&b->list, cap * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return CFPQ_ERR_NOMEM;
        }
        b->list_cap = cap;
    }
    ctl.list = b->list;
    ctl.list_cap = b->list_cap;
    ctl.k = k;
    ctl.max_rounds = max_rounds;
    ctl.any_jacobi = any_jacobi ? 1 : 0;
    ctl.limit_ns = (limit_ns > 0 && limit_ns < kLaunchLimitNs) ? limit_ns : kLaunchLimitNs;
    ctl.active = b->active;
    ctl.act = b->act;
    ctl.prod_off = b->prod_off;
    ctl.row_off = b->row_off;
    if (cudaMemcpyAsync(b->ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, s) != cudaSuccess) return CFPQ_ERR_CUDA;
    if (cudaMemcpyAsync(b->bq, hb, sizeof(BatchQuery) * k, cudaMemcpyHostToDevice, s) != cudaSuccess) return CFPQ_ERR_CUDA;
    if (cudaMemcpyAsync(b->active, active, sizeof(int) * k, cudaMemcpyHostToDevice, s) != cudaSuccess) return CFPQ_ERR_CUDA;
    return CFPQ_OK;
}

__global__ void k_collect_states(const BatchQuery *bq, int k, DevState *out) {
    const int j = blockIdx.x;
    if (j >= k) return;
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(bq[j].q.st);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(out + j);
    for (int w = threadIdx.x; w < (int)(sizeof(DevState) / 8); w += blockDim.x) dst[w] = __ldcg(src + w);
}
static_assert(sizeof(DevState) % 8 == 0, "DevState copied as 64-bit words");

int batch_collect_states(const BatchBuffers *b, const BatchQuery *d_bq, int k, cudaStream_t s) {
    k_collect_states<<<k, 128, 0, s>>>(d_bq, k, b->states);
    return cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

static std::mutex g_prof_mu;
static unsigned long long g_prof_ns[kBatchPhases], g_prof_rounds, g_prof_round_ns[kProfRounds];

void batch_record_profile(const BatchBuffers *b, cudaStream_t s) {
    BatchCtl ctl;
    if (cudaMemcpyAsync(&ctl, b->ctl, sizeof(ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    memcpy(g_prof_ns, ctl.phase_ns, sizeof(g_prof_ns));
    memcpy(g_prof_round_ns, ctl.round_product_ns, sizeof(g_prof_round_ns));
    g_prof_rounds = ctl.rounds;
}

void batch_buffers_free(BatchBuffers *b) {
    void *ptrs[] = {b->ctl, b->bq, b->active, b->act, b->prod_off, b->row_off, b->states, b->list};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    memset(b, 0, sizeof(*b));
}

}  // namespace cfpq

using namespace cfpq;

// Control buffers of batched solves, kept per device and grown on demand (no allocation
// or free, and so no device synchronisation, per call). Calls are serialised by the lock,
// which a solve holds until its launch has finished.
constexpr int kMaxBatchDevices = 64;
static std::mutex g_bufs_mu;
static BatchBuffers g_bufs[kMaxBatchDevices];

static int batch_buffers_for(int k, BatchBuffers **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxBatchDevices) return CFPQ_ERR_CUDA;
    BatchBuffers *b = &g_bufs[dev];
    if (b->k < k) {
        if (b->k) batch_buffers_free(b);
        const int rc = batch_buffers_alloc(b, std::max(k, 2 * b->k));
        if (rc != CFPQ_OK) return rc;
    }
    *out = b;
    return CFPQ_OK;
}

static int solve_grouped(cfpq_ctx *const *ctxs, int k, cudaStream_t s, const cfpq_batch_tuning &t, float *ms_out);

// One complete batched solve of ctxs under configuration t; *ms = device time of the batch
// (from its start on s until every query is solved). The queries of the size classes that
// t solves alone are begun first, each on its context's stream after s; the grouped launch
// takes the rest; s then waits for all of them.
static int solve_batch_with(cfpq_ctx *const *ctxs, int k, cudaStream_t s, const cfpq_batch_tuning &t, float *ms_out) {
    std::vector<cfpq_ctx *> grouped, alone;
    for (int j = 0; j < k; j++)
        (t.product[batch_size_class(ctxs[j]->W)] == CFPQ_BATCH_ALONE ? alone : grouped).push_back(ctxs[j]);
    if (alone.empty()) return solve_grouped(ctxs, k, s, t, ms_out);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreateWithFlags(&e0, cudaEventDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&e1, cudaEventDefault) != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return CFPQ_ERR_CUDA;
    }
    int rc = CFPQ_OK;
    size_t begun = 0;
    for (cfpq_ctx *c : alone) {
        if (cudaStreamWaitEvent(c->stream, e0, 0) != cudaSuccess) { rc = CFPQ_ERR_CUDA; break; }
        if ((rc = solve_begin(c, c->stream)) != CFPQ_OK) break;
        begun++;
    }
    if (rc == CFPQ_OK && !grouped.empty()) rc = solve_grouped(grouped.data(), (int)grouped.size(), s, t, nullptr);
    for (size_t j = 0; j < begun; j++)  // s waits for every solve begun (even after an error)
        if (cudaEventRecord(alone[j]->ev1, alone[j]->stream) != cudaSuccess ||
            cudaStreamWaitEvent(s, alone[j]->ev1, 0) != cudaSuccess)
            rc = CFPQ_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = CFPQ_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == CFPQ_ERR_CUDA) return rc;
    int worst = rc;  // the grouped launch's status (OK, or a limit some of its queries hit)
    for (size_t j = 0; j < begun; j++) {
        const int r = solve_end(alone[j], alone[j]->stream);
        if (r == CFPQ_ERR_CUDA) return r;
        if (r != CFPQ_OK && worst == CFPQ_OK) worst = r;
    }
    if (worst == CFPQ_OK && ms_out) *ms_out = ms;
    return worst;
}

// The grouped launch over ctxs; *ms = its device time.
static int solve_grouped(cfpq_ctx *const *ctxs, int k, cudaStream_t s, const cfpq_batch_tuning &t, float *ms_out) {
    std::lock_guard<std::mutex> lock(g_bufs_mu);
    std::vector<BatchQuery> hb(k);
    bool any_jacobi = false;
    for (int j = 0; j < k; j++) {
        fill_batch_query(ctxs[j], &hb[j], 1, t);
        any_jacobi |= hb[j].q.schedule == CFPQ_SCHED_JACOBI;
        ctxs[j]->solved = false;
        ctxs[j]->clean = false;
        ctxs[j]->last_stream = s;
        ctxs[j]->fixed_launches = 0;
        ctxs[j]->iter_launches = 0;
    }
    BatchBuffers *pb = nullptr;
    int rc = batch_buffers_for(k, &pb);
    if (rc != CFPQ_OK) return rc;
    BatchBuffers &bufs = *pb;
    std::vector<int> active(k, 1);
    // the smallest wall-clock limit among the contexts bounds the whole launch
    double limit_s = 0.0;
    for (int j = 0; j < k; j++)
        if (ctxs[j]->timeout_s > 0.0 && (limit_s == 0.0 || ctxs[j]->timeout_s < limit_s)) limit_s = ctxs[j]->timeout_s;
    if (rc == CFPQ_OK)
        rc = batch_buffers_upload(&bufs, hb.data(), active.data(), k, 1 << 30, any_jacobi, s,
                                  (unsigned long long)(limit_s * 1e9));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    if (rc == CFPQ_OK) rc = batch_launch(bufs.ctl, bufs.bq, s, t.blocks_per_sm, nullptr);
    cudaEventRecord(e1, s);
    unsigned err = 0;
    std::vector<DevState> states(k);
    if (rc == CFPQ_OK) rc = batch_collect_states(&bufs, bufs.bq, k, s);
    if (rc == CFPQ_OK && (cudaMemcpyAsync(&err, &bufs.ctl->error, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                          cudaMemcpyAsync(states.data(), bufs.states, sizeof(DevState) * k, cudaMemcpyDeviceToHost, s) !=
                              cudaSuccess))
        rc = CFPQ_ERR_CUDA;
    if (rc == CFPQ_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = CFPQ_ERR_CUDA;
    float ms = 0.f;
    if (rc == CFPQ_OK) {
        cudaEventElapsedTime(&ms, e0, e1);
        batch_record_profile(&bufs, s);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CFPQ_OK) return rc;
    if (err) return CFPQ_ERR_TIMEOUT;
    if (ms_out) *ms_out = ms;
    int worst = CFPQ_OK;
    for (int j = 0; j < k; j++) {
        const int r = apply_status(ctxs[j], states[j]);
        ctxs[j]->stats.solve_ms = ms;
        ctxs[j]->stats.schedule = hb[j].q.schedule;
        ctxs[j]->stats.gather_cpl = hb[j].cpl;
        ctxs[j]->stats.kernel_launches = 1;  // the whole batch is one cooperative launch
        ctxs[j]->solved = true;
        if (r == CFPQ_ERR_CUDA) return r;
        if (r != CFPQ_OK) worst = r;
    }
    return worst;
}

static int check_batch_args(cfpq_ctx *const *ctxs, int32_t k) {
    if (!ctxs || k <= 0 || k > kMaxBatch) return CFPQ_ERR_INVALID;
    for (int j = 0; j < k; j++)
        if (!ctxs[j] || ctxs[j]->block) return CFPQ_ERR_INVALID;  // a row block is solved with cfpq_block_*
    for (int j = 0; j < k; j++)
        if (ctxs[j]->lengths) return CFPQ_ERR_UNSUPPORTED;  // the grouped launch keeps no length planes
    return CFPQ_OK;
}

extern "C" void cfpq_batch_tuning_default(cfpq_batch_tuning *t) {
    if (!t) return;
    memset(t, 0, sizeof(*t));
    for (int c = 0; c < CFPQ_TUNE_CLASSES; c++) t->schedule[c] = CFPQ_SCHED_INPLACE;
}

extern "C" int cfpq_batch_tuning_get(cfpq_batch_tuning *t) {
    if (!t) return CFPQ_ERR_INVALID;
    batch_tuning_snapshot(t);
    return CFPQ_OK;
}

extern "C" int cfpq_batch_tuning_set(const cfpq_batch_tuning *t) {
    if (!t || !tuning_valid(*t)) return CFPQ_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune = *t;
    return CFPQ_OK;
}

extern "C" int cfpq_solve_batch(cfpq_ctx *const *ctxs, int32_t k, void *stream) {
    const int rc = check_batch_args(ctxs, k);
    if (rc != CFPQ_OK) return rc;
    cfpq_batch_tuning t;
    batch_tuning_snapshot(&t);
    return solve_batch_with(ctxs, k, stream ? (cudaStream_t)stream : ctxs[0]->stream, t, nullptr);
}

extern "C" int cfpq_solve_batch_tuned(cfpq_ctx *const *ctxs, int32_t k, const cfpq_batch_tuning *t, void *stream) {
    const int rc = check_batch_args(ctxs, k);
    if (rc != CFPQ_OK) return rc;
    if (!t || !tuning_valid(*t)) return CFPQ_ERR_INVALID;
    return solve_batch_with(ctxs, k, stream ? (cudaStream_t)stream : ctxs[0]->stream, *t, nullptr);
}

extern "C" int cfpq_autotune_batch(cfpq_ctx *const *ctxs, int32_t k, void *stream, cfpq_batch_tuning *best,
                                   cfpq_tune_report *report) {
    int rc = check_batch_args(ctxs, k);
    if (rc != CFPQ_OK) return rc;
    cudaStream_t s = stream ? (cudaStream_t)stream : ctxs[0]->stream;
    // size classes present, heaviest first (work ~ groups x rows x row words), and the
    // classes holding contexts whose schedule is the library's choice
    std::vector<double> work(CFPQ_TUNE_CLASSES, 0.0);
    std::vector<bool> has_auto(CFPQ_TUNE_CLASSES, false);
    for (int j = 0; j < k; j++) {
        const int c = batch_size_class(ctxs[j]->W);
        work[c] += (double)ctxs[j]->n_groups * ctxs[j]->n * ctxs[j]->W;
        if (ctxs[j]->schedule_req == CFPQ_SCHED_AUTO) has_auto[c] = true;
    }
    std::vector<int> classes;
    for (int c = 0; c < CFPQ_TUNE_CLASSES; c++)
        if (work[c] > 0.0) classes.push_back(c);
    std::sort(classes.begin(), classes.end(), [&](int a, int b) { return work[a] > work[b]; });

    int trials = 0;
    auto timed = [&](const cfpq_batch_tuning &t, float *ms) {
        trials++;
        return solve_batch_with(ctxs, k, s, t, ms);
    };
    cfpq_batch_tuning cur;
    cfpq_batch_tuning_default(&cur);
    float cur_ms = 0.f;
    rc = timed(cur, &cur_ms);
    if (rc != CFPQ_OK) return rc;
    const float default_ms = cur_ms;
    auto consider = [&](const cfpq_batch_tuning &cand) -> int {
        float ms = 0.f;
        const int r = timed(cand, &ms);
        if (r != CFPQ_OK) return r;
        if (ms < 0.97f * cur_ms) {
            cur = cand;
            cur_ms = ms;
        }
        return CFPQ_OK;
    };
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, 256, 0) != cudaSuccess || per_sm < 1)
        return CFPQ_ERR_CUDA;
    for (int bps : {1, 2, 4, 8}) {
        if (bps > per_sm || bps == std::min(per_sm, 8)) continue;  // the default is already timed
        cfpq_batch_tuning cand = cur;
        cand.blocks_per_sm = bps;
        if ((rc = consider(cand)) != CFPQ_OK) return rc;
    }
    for (int c : classes) {
        int builtin = 1;
        gather_chunks(1u << c, &builtin);
        const int now = cur.cpl[c] > 0 ? cur.cpl[c] : builtin;
        for (int v : {1, 2, 4, 8}) {
            if (v == now) continue;
            cfpq_batch_tuning cand = cur;
            cand.cpl[c] = v;
            if ((rc = consider(cand)) != CFPQ_OK) return rc;
        }
    }
    for (int c : classes) {
        if (!has_auto[c]) continue;
        cfpq_batch_tuning cand = cur;
        cand.schedule[c] = cur.schedule[c] == CFPQ_SCHED_INPLACE ? CFPQ_SCHED_JACOBI : CFPQ_SCHED_INPLACE;
        if ((rc = consider(cand)) != CFPQ_OK) return rc;
    }
    // classes of queries whose own tiles come close to filling the GPU (W > 32 words: n_pad >
    // 1024) may be solved alone beside the launch, with tensor-core products where they pay
    for (int c : classes) {
        if (c < 6) continue;
        cfpq_batch_tuning cand = cur;
        cand.product[c] = CFPQ_BATCH_ALONE;
        if ((rc = consider(cand)) != CFPQ_OK) return rc;
    }
    // confirm (the contexts end with the chosen configuration's results and statistics)
    float best_ms = 0.f;
    if ((rc = timed(cur, &best_ms)) != CFPQ_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune.blocks_per_sm = cur.blocks_per_sm;
        for (int c : classes) {
            g_tune.cpl[c] = cur.cpl[c];
            g_tune.product[c] = cur.product[c];
            if (has_auto[c]) g_tune.schedule[c] = cur.schedule[c];
        }
    }
    if (best) *best = cur;
    if (report) {
        report->trials = trials;
        report->default_ms = default_ms;
        report->best_ms = best_ms;
    }
    return CFPQ_OK;
}

extern "C" int cfpq_batch_last_profile(double *phase_ms, int32_t n_phases, int64_t *rounds,
                                       double *round_product_ms, int32_t n_round_slots) {
    if ((!phase_ms && n_phases > 0) || n_phases < 0) return CFPQ_ERR_INVALID;
    if ((!round_product_ms && n_round_slots > 0) || n_round_slots < 0) return CFPQ_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    for (int i = 0; i < n_phases; i++) phase_ms[i] = i < kBatchPhases ? (double)g_prof_ns[i] * 1e-6 : 0.0;
    for (int i = 0; i < n_round_slots; i++)
        round_product_ms[i] = (i < kProfRounds && (uint64_t)i < g_prof_rounds) ? (double)g_prof_round_ns[i] * 1e-6 : 0.0;
    if (rounds) *rounds = (int64_t)g_prof_rounds;
    return CFPQ_OK;
}
