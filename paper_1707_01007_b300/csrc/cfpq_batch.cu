// Batched closure: many independent queries advanced together by one persistent
// (cooperative) launch. Each round performs one execution of Algorithm 1's loop body
// (Section 4.2) for every query that has not converged; a query whose round added no
// pair is retired while the others continue (per-query convergence). All queries share
// the grid: work items (query, production group, row, column chunk) are spread over
// all warps, so small and large queries overlap on the device.
//
// Every wait in this file (the grid barrier) is bounded by a %globaltimer deadline;
// on expiry the kernel records an error and returns.
#include <algorithm>
#include <cstring>
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
        ctl->prod_off[A] = P;
        ctl->row_off[A] = R;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_batch(BatchCtl *ctl, const BatchQuery *bq) {
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gwarp = gtid >> 5, gwarps = gthreads >> 5;
    const int lane = threadIdx.x & 31;
    const int k = ctl->k;
    if (gtid == 0) ctl->start_ns = globaltimer_ns();

    // 1) queries starting in this launch: clear their matrices and state
    for (int j = 0; j < k; j++) {
        if (!bq[j].init) continue;
        const QDesc &q = bq[j].q;
        const uint64_t words = (uint64_t)q.n_nt * q.plane;
        uint4 *p4[3] = {(uint4 *)q.T, (uint4 *)q.X0, (uint4 *)q.X1};
        for (int b = 0; b < 3; b++)
            for (uint64_t w = gtid; w < words / 4; w += gthreads) p4[b][w] = make_uint4(0, 0, 0, 0);
        const uint64_t rw = (uint64_t)q.n_nt * q.W;
        for (uint64_t w = gtid; w < rw; w += gthreads) {
            q.R0[w] = 0;
            q.R1[w] = 0;
            q.Trow[w] = 0;
        }
        if (gtid == 0) {
            DevState *st = q.st;
            const unsigned long long mi = st->max_iter;
            memset(st, 0, sizeof(DevState));
            st->max_iter = mi;
            for (int a = 0; a < q.n_nt; a++) st->dirty[a] = 1u;
        }
    }
    if (!grid_barrier(ctl)) return;
    // 2) matrix initialisation of the new queries
    for (int j = 0; j < k; j++)
        if (bq[j].init) seed_query(bq[j].q, gtid, gthreads);
    if (!grid_barrier(ctl)) return;
    if (blockIdx.x == 0) build_tables(ctl, bq, 0);
    if (!grid_barrier(ctl)) return;

    for (int round = 0; round < ctl->max_rounds; round++) {
        const int na = min((int)ld_u32(&ctl->n_active), k);
        if (na <= 0) break;
        // 3) products of every active query
        const unsigned long long np = __ldcg(ctl->prod_off + na);
        for (unsigned long long it = gwarp; it < np; it += gwarps) {
            const int s = find_slot(ctl->prod_off, na, it);
            const int j = __ldcg(ctl->act + s);
            if (j < 0 || j >= k) continue;
            const BatchQuery &b = bq[j];
            const unsigned long long loc = it - __ldcg(ctl->prod_off + s);
            const unsigned long long per_group = (unsigned long long)b.q.n * b.nch;
            const unsigned long long g64 = loc / per_group;
            const unsigned long long r = loc % per_group;
            const uint32_t i = (uint32_t)(r / b.nch), ch = (uint32_t)(r % b.nch);
            if (g64 >= (unsigned long long)b.q.n_groups || i >= b.q.n) continue;
            const int g = (int)g64;
            const uint32_t parity = (uint32_t)(ld_u64(&b.q.st->iter) & 1ull);
            switch (b.cpl) {
                case 1: gather_row_chunk<1>(b.q, g, i, ch, lane, parity); break;
                case 2: gather_row_chunk<2>(b.q, g, i, ch, lane, parity); break;
                case 4: gather_row_chunk<4>(b.q, g, i, ch, lane, parity); break;
                default: gather_row_chunk<8>(b.q, g, i, ch, lane, parity); break;
            }
        }
        if (!grid_barrier(ctl)) return;
        const unsigned long long nr = __ldcg(ctl->row_off + na);
        // 4) Jacobi queries: T |= N
        if (ctl->any_jacobi) {
            for (unsigned long long it = gwarp; it < nr; it += gwarps) {
                const int s = find_slot(ctl->row_off, na, it);
                const int j = __ldcg(ctl->act + s);
                if (j < 0 || j >= k) continue;
                const BatchQuery &b = bq[j];
                if (b.q.schedule != CFPQ_SCHED_JACOBI) continue;
                const unsigned long long loc = it - __ldcg(ctl->row_off + s);
                if (loc >= b.row_items) continue;
                merge_row(b.q, (int)(loc / b.q.n), (uint32_t)(loc % b.q.n), lane,
                          (uint32_t)(ld_u64(&b.q.st->iter) & 1ull));
            }
            if (!grid_barrier(ctl)) return;
        }
        // 5) clear the delta plane that was read
        for (unsigned long long it = gwarp; it < nr; it += gwarps) {
            const int s = find_slot(ctl->row_off, na, it);
            const int j = __ldcg(ctl->act + s);
            if (j < 0 || j >= k) continue;
            const BatchQuery &b = bq[j];
            const unsigned long long loc = it - __ldcg(ctl->row_off + s);
            if (loc >= b.row_items) continue;
            clear_row(b.q, (int)(loc / b.q.n), (uint32_t)(loc % b.q.n), lane, (uint32_t)(ld_u64(&b.q.st->iter) & 1ull));
        }
        if (!grid_barrier(ctl)) return;
        // 6) per-query end of iteration; a converged query is retired
        for (int s = blockIdx.x; s < na; s += gridDim.x) {
            const int j = __ldcg(ctl->act + s);
            if (j < 0 || j >= k) continue;  // uniform across the block
            const unsigned cont = tail_query(bq[j].q, threadIdx.x, blockDim.x);
            if (threadIdx.x == 0) {
                bq[j].q.st->gather_products += (unsigned long long)bq[j].q.n_rules;
                if (!cont) ctl->active[j] = 0;
            }
            __syncthreads();
        }
        // every tail must be done (it reads act[] and writes active[]) before the tables change
        if (!grid_barrier(ctl)) return;
        if (blockIdx.x == 0) {
            build_tables(ctl, bq, round + 1);
            if (threadIdx.x == 0 && ctl->limit_ns && globaltimer_ns() - ctl->start_ns > ctl->limit_ns)
                atomicExch(&ctl->error, 2u);
            __syncthreads();
        }
        if (!grid_barrier(ctl)) return;
    }
}

int batch_launch(BatchCtl *d_ctl, const BatchQuery *d_bq, cudaStream_t s, int *grid_out) {
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CFPQ_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return CFPQ_ERR_UNSUPPORTED;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, 256, 0) != cudaSuccess || per_sm < 1)
        return CFPQ_ERR_CUDA;
    const int grid = sms * std::min(per_sm, 8);
    void *args[] = {(void *)&d_ctl, (void *)&d_bq};
    if (cudaLaunchCooperativeKernel((const void *)k_batch, dim3(grid), dim3(256), args, 0, s) != cudaSuccess)
        return CFPQ_ERR_CUDA;
    if (grid_out) *grid_out = grid;
    return CFPQ_OK;
}

void fill_batch_query(const cfpq_ctx *c, BatchQuery *b, int init) {
    memset(b, 0, sizeof(*b));
    b->q = c->hq;
    int cpl = 1;
    const uint32_t nch = gather_chunks(c->W, &cpl);
    b->cpl = cpl;
    b->nch = nch;
    b->prod_items = (unsigned long long)c->n_groups * c->n * nch;
    b->row_items = (unsigned long long)c->n_nt * c->n;
    b->init = init;
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
        cudaMalloc(&b->row_off, sizeof(unsigned long long) * (k + 1)) != cudaSuccess) {
        cudaGetLastError();
        batch_buffers_free(b);
        return CFPQ_ERR_NOMEM;
    }
    return CFPQ_OK;
}

int batch_buffers_upload(BatchBuffers *b, const BatchQuery *hb, const int *active, int k, int max_rounds,
                         bool any_jacobi, cudaStream_t s) {
    BatchCtl ctl;
    memset(&ctl, 0, sizeof(ctl));
    ctl.k = k;
    ctl.max_rounds = max_rounds;
    ctl.any_jacobi = any_jacobi ? 1 : 0;
    ctl.limit_ns = kLaunchLimitNs;
    ctl.active = b->active;
    ctl.act = b->act;
    ctl.prod_off = b->prod_off;
    ctl.row_off = b->row_off;
    if (cudaMemcpyAsync(b->ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, s) != cudaSuccess) return CFPQ_ERR_CUDA;
    if (cudaMemcpyAsync(b->bq, hb, sizeof(BatchQuery) * k, cudaMemcpyHostToDevice, s) != cudaSuccess) return CFPQ_ERR_CUDA;
    if (cudaMemcpyAsync(b->active, active, sizeof(int) * k, cudaMemcpyHostToDevice, s) != cudaSuccess) return CFPQ_ERR_CUDA;
    return CFPQ_OK;
}

void batch_buffers_free(BatchBuffers *b) {
    void *ptrs[] = {b->ctl, b->bq, b->active, b->act, b->prod_off, b->row_off};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    memset(b, 0, sizeof(*b));
}

}  // namespace cfpq

using namespace cfpq;

extern "C" int cfpq_solve_batch(cfpq_ctx *const *ctxs, int32_t k, void *stream) {
    if (!ctxs || k <= 0) return CFPQ_ERR_INVALID;
    for (int j = 0; j < k; j++)
        if (!ctxs[j]) return CFPQ_ERR_INVALID;
    cudaStream_t s = stream ? (cudaStream_t)stream : ctxs[0]->stream;
    std::vector<BatchQuery> hb(k);
    bool any_jacobi = false;
    for (int j = 0; j < k; j++) {
        fill_batch_query(ctxs[j], &hb[j], 1);
        any_jacobi |= ctxs[j]->schedule == CFPQ_SCHED_JACOBI;
        ctxs[j]->solved = false;
        ctxs[j]->last_stream = s;
        ctxs[j]->fixed_launches = 0;
        ctxs[j]->iter_launches = 0;
    }
    BatchBuffers bufs;
    int rc = batch_buffers_alloc(&bufs, k);
    if (rc != CFPQ_OK) return rc;
    // the per-query state carries each query's iteration cap into the kernel
    for (int j = 0; j < k && rc == CFPQ_OK; j++) {
        DevState st0;
        memset(&st0, 0, sizeof(st0));
        st0.max_iter = ctxs[j]->max_iter;
        if (cudaMemcpyAsync(ctxs[j]->d_state, &st0, sizeof(st0), cudaMemcpyHostToDevice, s) != cudaSuccess)
            rc = CFPQ_ERR_CUDA;
    }
    std::vector<int> active(k, 1);
    if (rc == CFPQ_OK) rc = batch_buffers_upload(&bufs, hb.data(), active.data(), k, 1 << 30, any_jacobi, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    if (rc == CFPQ_OK) rc = batch_launch(bufs.ctl, bufs.bq, s, nullptr);
    cudaEventRecord(e1, s);
    unsigned err = 0;
    if (rc == CFPQ_OK && cudaMemcpyAsync(&err, &bufs.ctl->error, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = CFPQ_ERR_CUDA;
    if (rc == CFPQ_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = CFPQ_ERR_CUDA;
    float ms = 0.f;
    if (rc == CFPQ_OK) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    batch_buffers_free(&bufs);
    if (rc != CFPQ_OK) return rc;
    if (err) return CFPQ_ERR_TIMEOUT;
    int worst = CFPQ_OK;
    for (int j = 0; j < k; j++) {
        const int r = read_status(ctxs[j], s);
        ctxs[j]->stats.solve_ms = ms;
        ctxs[j]->stats.kernel_launches = 1;  // the whole batch is one cooperative launch
        ctxs[j]->solved = true;
        if (r == CFPQ_ERR_CUDA) return r;
        if (r != CFPQ_OK) worst = r;
    }
    return worst;
}
