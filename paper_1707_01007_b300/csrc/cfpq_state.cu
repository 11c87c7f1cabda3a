// Checkpoint and resume of the fixpoint loop (cfpq_state_size, cfpq_export_state,
// cfpq_import_state, cfpq_resume).
//
// After k executions of Algorithm 1's loop (Section 4.2), everything the next execution
// needs is T_k itself and the pairs the k-th execution added (the semi-naive delta the
// gather reads; a tensor-core execution joins all of T), with their row bitmaps and counts.
// The closure is monotone and its least fixpoint unique (Theorem 2), so continuing from a
// saved T_k and its delta reaches the same result as an uninterrupted solve, and under the
// Jacobi schedule after the same total number of executions. Everything else is rebuilt
// on resume: the transposes and tile occupancy of the operands, and the gather list of the
// next execution.
//
// State image (host memory): a header, then T (n_nt planes of n_pad rows x W words), the
// delta plane of the next execution, its row bitmap, T's row bitmap and T's word summary.
#include <cstring>
#include <vector>

#include "cfpq_internal.h"

namespace cfpq {

__global__ void __launch_bounds__(256) k_scan_rows(const QDesc *qd, uint32_t *list, uint32_t cap,
                                                  uint32_t nch);  // cfpq_api.cu

namespace {

constexpr uint64_t kMagic = 0x4154535150464343ull;  // "CCFPQSTA"
constexpr uint32_t kVersion = 1;

struct StateHeader {
    uint64_t magic;
    uint32_t version, n, n_pad, n_nt, n_rules, schedule, SW, pad;
    uint64_t rules_hash;
    uint64_t iter, new_bits, seed_bits, tensor_products, gather_products;
    uint64_t tcount[kMaxNT], dcount[kMaxNT];  // pairs in T[A]; in the delta the next execution reads
};

// FNV-1a over the deduplicated productions and the counts that fix the image's layout.
uint64_t rules_hash(const cfpq_ctx *c) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint32_t v) {
        for (int b = 0; b < 4; b++) {
            h ^= (v >> (8 * b)) & 0xFFu;
            h *= 1099511628211ull;
        }
    };
    mix((uint32_t)c->n_nt);
    mix((uint32_t)c->n_unary);
    mix((uint32_t)c->n_eps_rules);
    for (const Rule &r : c->rules) {
        mix((uint32_t)r.lhs);
        mix((uint32_t)r.b);
        mix((uint32_t)r.c);
    }
    return h;
}

size_t plane_bytes(const cfpq_ctx *c) { return (size_t)c->n_nt * c->plane * sizeof(uint32_t); }
size_t rows_bytes(const cfpq_ctx *c) { return (size_t)c->n_nt * c->W * sizeof(uint32_t); }
size_t sum_bytes(const cfpq_ctx *c) { return (size_t)c->n_nt * c->n_pad * c->SW * sizeof(uint32_t); }

size_t image_bytes(const cfpq_ctx *c) {
    return sizeof(StateHeader) + 2 * plane_bytes(c) + 2 * rows_bytes(c) + sum_bytes(c);
}

// Contexts whose loop state is T and one delta plane: matrix paths without lengths, not a
// row block of a sharded solve.
bool checkpointable(const cfpq_ctx *c) {
    return c->path != CFPQ_PATH_WORKLIST && !c->lengths && !c->block && c->n_groups > 0;
}

}  // namespace
}  // namespace cfpq

using namespace cfpq;

// a failed CUDA call ends the entry point with CFPQ_ERR_CUDA
#define CK(call)                                   \
    do {                                           \
        if ((call) != cudaSuccess) {               \
            cudaGetLastError();                    \
            return CFPQ_ERR_CUDA;                  \
        }                                          \
    } while (0)

extern "C" int cfpq_state_size(const cfpq_ctx *c, size_t *bytes) {
    if (!c || !bytes) return CFPQ_ERR_INVALID;
    if (!checkpointable(c)) return CFPQ_ERR_UNSUPPORTED;
    *bytes = image_bytes(c);
    return CFPQ_OK;
}

extern "C" int cfpq_export_state(cfpq_ctx *c, void *buf, size_t cap) {
    if (!c || !buf) return CFPQ_ERR_INVALID;
    if (!checkpointable(c)) return CFPQ_ERR_UNSUPPORTED;
    if (!c->solved) return CFPQ_ERR_NOT_SOLVED;
    if (c->switched) return CFPQ_ERR_UNSUPPORTED;  // finished by the worklist path: no delta plane
    if (cap < image_bytes(c)) return CFPQ_ERR_BUFFER;
    cudaStream_t s = c->last_stream ? c->last_stream : c->stream;
    DevState st;
    CK(cudaMemcpyAsync(&st, c->d_state, sizeof(st), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint32_t p = (uint32_t)(st.iter & 1ull);  // the plane the next execution reads
    StateHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = kMagic;
    h.version = kVersion;
    h.n = c->n;
    h.n_pad = c->n_pad;
    h.n_nt = (uint32_t)c->n_nt;
    h.n_rules = (uint32_t)c->rules.size();
    h.schedule = (uint32_t)c->schedule;
    h.SW = c->SW;
    h.rules_hash = rules_hash(c);
    h.iter = st.iter;
    h.new_bits = st.new_bits;
    h.seed_bits = st.seed_bits;
    h.tensor_products = st.tensor_products;
    h.gather_products = st.gather_products;
    for (int a = 0; a < c->n_nt; a++) {
        h.tcount[a] = st.tcount[a];
        h.dcount[a] = st.dcount[p][a];
    }
    char *out = static_cast<char *>(buf);
    memcpy(out, &h, sizeof(h));
    size_t off = sizeof(h);
    auto down = [&](const void *src, size_t bytes) -> bool {
        if (cudaMemcpyAsync(out + off, src, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
        off += bytes;
        return true;
    };
    const bool ok = down(c->d_T, plane_bytes(c)) && down(p ? c->d_X1 : c->d_X0, plane_bytes(c)) &&
                    down(p ? c->d_R1 : c->d_R0, rows_bytes(c)) && down(c->d_Trow, rows_bytes(c)) &&
                    down(c->d_Tsum, sum_bytes(c));
    if (!ok) return CFPQ_ERR_CUDA;
    CK(cudaStreamSynchronize(s));
    return CFPQ_OK;
}

extern "C" int cfpq_import_state(cfpq_ctx *c, const void *buf, size_t bytes) {
    if (!c || !buf) return CFPQ_ERR_INVALID;
    if (!checkpointable(c)) return CFPQ_ERR_UNSUPPORTED;
    if (bytes < sizeof(StateHeader)) return CFPQ_ERR_INVALID;
    StateHeader h;
    memcpy(&h, buf, sizeof(h));
    if (h.magic != kMagic || h.version != kVersion || h.n != c->n || h.n_pad != c->n_pad ||
        h.n_nt != (uint32_t)c->n_nt || h.n_rules != (uint32_t)c->rules.size() || h.SW != c->SW ||
        h.rules_hash != rules_hash(c) || bytes != image_bytes(c))
        return CFPQ_ERR_INVALID;
    cudaStream_t s = c->stream;
    const uint32_t p = (uint32_t)(h.iter & 1ull);
    const char *in = static_cast<const char *>(buf);
    size_t off = sizeof(h);
    auto up = [&](void *dst, size_t n) -> bool {
        if (cudaMemcpyAsync(dst, in + off, n, cudaMemcpyHostToDevice, s) != cudaSuccess) return false;
        off += n;
        return true;
    };
    const bool ok = up(c->d_T, plane_bytes(c)) && up(p ? c->d_X1 : c->d_X0, plane_bytes(c)) &&
                    up(p ? c->d_R1 : c->d_R0, rows_bytes(c)) && up(c->d_Trow, rows_bytes(c)) &&
                    up(c->d_Tsum, sum_bytes(c));
    if (!ok) return CFPQ_ERR_CUDA;
    // the delta plane the next execution writes starts empty
    CK(cudaMemsetAsync(p ? c->d_X0 : c->d_X1, 0, plane_bytes(c), s));
    CK(cudaMemsetAsync(p ? c->d_R0 : c->d_R1, 0, rows_bytes(c), s));
    DevState st;
    memset(&st, 0, sizeof(st));
    st.iter = h.iter;
    st.max_iter = c->max_iter;
    st.new_bits = h.new_bits;
    st.seed_bits = h.seed_bits;
    st.tensor_products = h.tensor_products;
    st.gather_products = h.gather_products;
    for (int a = 0; a < c->n_nt; a++) {
        st.tcount[a] = h.tcount[a];
        st.dcount[p][a] = h.dcount[a];
        st.dirty[a] = st.occ_now[a] = 1u;  // transposes and tile occupancy are rebuilt
    }
    for (int g = 0; g < c->n_groups && g < kMaxNT; g++) st.use_tensor[g] = c->group_tensor[g] ? 1u : 0u;
    CK(cudaMemcpyAsync(c->d_state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    c->clean = false;
    c->switched = false;
    c->resumable = true;
    c->solved = false;
    return CFPQ_OK;
}

extern "C" int cfpq_resume(cfpq_ctx *c, void *stream, int64_t more_executions) {
    if (!c || more_executions < 0) return CFPQ_ERR_INVALID;
    if (!checkpointable(c)) return CFPQ_ERR_UNSUPPORTED;
    if (!c->resumable) return CFPQ_ERR_NOT_SOLVED;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    c->solved = false;
    c->last_stream = s;
    c->stats.product_ms = c->stats.tensor_ms = c->stats.lengths_ms = 0.0;
    c->stats.product_launches = c->stats.tensor_launches = c->stats.lengths_launches = 0;
    CK(cudaEventRecord(c->ev0, s));
    // the loop's flags start afresh; the cap counts from here (or is the context's own)
    DevState st;
    CK(cudaMemcpyAsync(&st, c->d_state, sizeof(st), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st.error = st.done = st.cont = st.changed = 0u;
    st.loop_go = 0u;
    st.gbar = 0ull;
    st.small_run = st.to_worklist = 0u;
    st.skip = st.any_next = 0u;  // the graph loop's flags (the first execution of a loop iteration runs regardless)
    // 0: Theorem 3's bound on changing executions, |V|^2 |N|, plus the final one
    const double bound = (double)c->n * (double)c->n * (double)c->n_nt + 1.0;
    st.max_iter = more_executions > 0 ? st.iter + (uint64_t)more_executions
                                      : (bound > 1.8e19 ? ~0ull : (uint64_t)bound);
    st.deadline_ns = 0;
    st.list_len[0] = st.list_len[1] = 0u;
    for (int a = 0; a < c->n_nt; a++) st.dirty[a] = st.occ_now[a] = 1u;
    for (int g = 0; g < c->n_groups && g < kMaxNT; g++) st.use_tensor[g] = c->group_tensor[g] ? 1u : 0u;
    for (int g = 0; g < kMaxNT; g++) st.plan_count[g][0] = st.plan_count[g][1] = st.plan_take[g][0] =
        st.plan_take[g][1] = 0u;
    CK(cudaMemcpyAsync(c->d_state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
    c->fixed_launches = 0;
    if (c->timeout_s > 0) {
        arm_deadline(c, s);
        c->fixed_launches++;
    }
    if (c->any_gather) {  // the gather list of the next execution, from the delta just restored
        int cpl;
        const uint32_t nch = gather_chunks(c->W, &cpl);
        const uint64_t items = (uint64_t)c->n_groups * ((c->n + 31) / 32);
        k_scan_rows<<<(uint32_t)((items + 255) / 256), 256, 0, s>>>(c->d_q, c->d_list, c->list_cap, nch);
        CK(cudaGetLastError());
        c->fixed_launches++;
    }
    bool any_tensor = false;
    for (int g = 0; g < c->n_groups; g++) any_tensor |= c->group_tensor[g] != 0;
    int rc = any_tensor ? enqueue_tensor_seed_transposes(c, s, &c->fixed_launches) : CFPQ_OK;
    if (rc != CFPQ_OK) return rc;
    if ((rc = run_loop(c, s)) != CFPQ_OK) return rc;
    CK(cudaEventRecord(c->ev1, s));
    rc = solve_end(c, s);
    // an interrupted solve can be resumed again; a finished one cannot
    c->resumable = rc == CFPQ_ERR_ITER_LIMIT || rc == CFPQ_ERR_TIMEOUT;
    return rc;
}
