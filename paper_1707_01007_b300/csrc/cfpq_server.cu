// Serving: continuous batching of independent CFPQ queries on one GPU.
//
// Queries are submitted at any time and wait in a FIFO. Each cfpq_server_step
//   1. admits waiting queries in order while their device footprint (the bit-packed
//      matrices of Algorithm 1's closure, Section 4.2, plus delta planes and bookkeeping)
//      fits in the free part of the HBM budget; a query larger than the whole budget
//      fails with NOMEM;
//   2. runs one persistent grouped launch (the batched kernel) that zeroes and seeds the
//      newly admitted queries and then advances every resident query by up to
//      `rounds_per_step` loop executions; queries of every size share the grid, so their
//      work overlaps on the device;
//   3. retires the queries whose loop stopped (fixpoint or iteration cap): their R_A are
//      copied to host memory and their device memory goes back to the stream-ordered
//      pool at once, so the next step can admit more.
// Large queries (n_pad >= kSoloRows) do not join the grouped launch: one large query's round
// and the clearing of its planes would lengthen the step of every small query resident with
// it, and the single-query loop (a CUDA graph with a conditional while node) runs a large
// query several times faster than the grouped launch does. They are solved on a second
// stream by that loop, concurrently with the grouped launches; each step polls their
// completion events and retires the finished ones in the same way.
// Results are identical to solving each query alone: each query runs Algorithm 1 to its
// own least fixpoint; other queries only share the launch.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "cfpq_batch.h"
#include "cfpq_internal.h"

using namespace cfpq;

namespace {

struct Pending {
    int64_t ticket;
    int32_t n_nt, n_term;
    uint32_t n;
    std::vector<cfpq_rule1> unary;
    std::vector<cfpq_rule2> binary;
    std::vector<int32_t> eps;
    std::vector<cfpq_edge> edges;
    size_t footprint;
    int schedule;
};

struct Served {
    int64_t ticket = 0;
    cfpq_ctx *ctx = nullptr;
    bool solo = false;  // solved by the single-query loop on the server's second stream
    size_t footprint = 0;
    int state = CFPQ_QUERY_QUEUED;
    int status = CFPQ_OK;
    int init = 1;
    int64_t iterations = 0;
    std::vector<std::vector<cfpq_triple>> results;  // per non-terminal, sorted (m, n)
};

}  // namespace

constexpr uint32_t kSoloRows = 16384;  // queries with at least this many (padded) rows run alone

struct cfpq_server {
    size_t budget = 0, used = 0, peak_used = 0;
    int rounds = 8, max_resident = 4096;
    cudaStream_t stream = nullptr;
    cudaStream_t solo_stream = nullptr;  // large queries' single-query loops
    std::vector<Served *> solo;          // large queries in flight there
    cudaMemPool_t pool = nullptr;
    std::deque<Pending> waiting;
    std::vector<Served *> resident;
    std::map<int64_t, Served *> finished;
    std::map<int64_t, int> state_of;  // every ticket ever issued and not released
    int64_t next_ticket = 1;
    BatchBuffers bufs{};
    int bufs_cap = 0;
    int64_t launches = 0, steps = 0, completed = 0, failed = 0;
    double admit_ms = 0.0, launch_ms = 0.0, retire_ms = 0.0;  // host wall time per phase of the steps
    std::vector<int64_t> just_finished;  // tickets finished since the last cfpq_server_completed
    // page-locked staging of a step's retirements: loop states, per-non-terminal offsets, triples
    DevState *h_state = nullptr;
    unsigned long long *h_off = nullptr;
    cfpq_triple *h_trip = nullptr;
    size_t state_cap = 0, off_cap = 0, trip_cap = 0;
};

// Page-locked host array of at least `need` elements (grown by half again; the old one freed).
template <class T>
static bool host_reserve(T *&p, size_t &cap, size_t need) {
    if (cap >= need) return true;
    if (p) cudaFreeHost(p);
    p = nullptr;
    const size_t n = std::max<size_t>(need, cap + cap / 2);
    cap = 0;
    if (cudaHostAlloc(reinterpret_cast<void **>(&p), std::max<size_t>(n, 1) * sizeof(T), cudaHostAllocDefault) !=
        cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return false;
    }
    cap = n;
    return true;
}

static int server_bufs(cfpq_server *s, int k) {
    if (k <= s->bufs_cap) return CFPQ_OK;
    if (s->bufs_cap) batch_buffers_free(&s->bufs);
    int cap = std::max(k, 2 * s->bufs_cap);
    const int rc = batch_buffers_alloc(&s->bufs, cap);
    s->bufs_cap = rc == CFPQ_OK ? cap : 0;
    return rc;
}

extern "C" int cfpq_server_options_default(cfpq_server_options *o) {
    if (!o) return CFPQ_ERR_INVALID;
    memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = 0;
    o->rounds_per_step = 8;
    o->max_resident = 4096;
    return CFPQ_OK;
}

extern "C" int cfpq_server_create(const cfpq_server_options *opt, cfpq_server **out) {
    if (!out) return CFPQ_ERR_INVALID;
    cfpq_server_options o;
    cfpq_server_options_default(&o);
    if (opt) o = *opt;
    if (o.rounds_per_step < 0 || o.max_resident < 0 || o.max_resident > kMaxBatch) return CFPQ_ERR_INVALID;
    cfpq_server *s = new (std::nothrow) cfpq_server();
    if (!s) return CFPQ_ERR_NOMEM;
    s->rounds = o.rounds_per_step ? o.rounds_per_step : 8;
    s->max_resident = o.max_resident ? o.max_resident : 4096;
    int dev = 0;
    size_t free_b = 0, total_b = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->solo_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaDeviceGetDefaultMemPool(&s->pool, dev) != cudaSuccess) {
        cudaGetLastError();
        if (s->stream) cudaStreamDestroy(s->stream);
        if (s->solo_stream) cudaStreamDestroy(s->solo_stream);
        delete s;
        return CFPQ_ERR_CUDA;
    }
    // keep freed query memory in the pool for the next admissions instead of returning it
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    s->budget = o.hbm_budget_bytes ? (size_t)o.hbm_budget_bytes : (size_t)(0.9 * (double)free_b);
    *out = s;
    return CFPQ_OK;
}

extern "C" int cfpq_server_submit(cfpq_server *s, const cfpq_grammar_cnf *g, uint32_t n, const cfpq_edge *edges,
                                  size_t n_edges, int32_t schedule, int64_t *ticket) {
    if (!s || !ticket) return CFPQ_ERR_INVALID;
    cfpq_options o;
    cfpq_options_default(&o);
    o.schedule = schedule;
    const int rc = validate_inputs(g, n, edges, n_edges, &o);
    if (rc != CFPQ_OK) return rc;
    Pending p;
    p.ticket = s->next_ticket++;
    p.n_nt = g->n_nonterm;
    p.n_term = g->n_term;
    p.n = n;
    p.unary.assign(g->unary, g->unary + g->n_unary);
    p.binary.assign(g->binary, g->binary + g->n_binary);
    p.eps.assign(g->eps_lhs, g->eps_lhs + g->n_eps);
    p.edges.assign(edges, edges + n_edges);
    p.footprint = query_footprint(n, g->n_nonterm, n_edges, g->n_binary, false);
    p.schedule = schedule;
    s->state_of[p.ticket] = CFPQ_QUERY_QUEUED;
    *ticket = p.ticket;
    s->waiting.push_back(std::move(p));
    return CFPQ_OK;
}

// Copies every R_A of the stopped queries qs (all on stream st) to the host and returns their
// device memory. Two waits for the whole set: one for every query's loop state and relation
// sizes (the counting kernels of all queries enqueued first), one for the triples of all of
// them, emitted and copied into page-locked staging back to back. On an error nothing has
// been freed yet (the caller keeps the queries).
static int retire_batch(cfpq_server *s, const std::vector<Served *> &qs, cudaStream_t st) {
    const size_t k = qs.size();
    if (k == 0) return CFPQ_OK;
    size_t n_off = 0;
    for (Served *q : qs) n_off += (size_t)q->ctx->n_nt + 1;
    if (!host_reserve(s->h_state, s->state_cap, k) || !host_reserve(s->h_off, s->off_cap, n_off)) return CFPQ_ERR_NOMEM;
    std::vector<size_t> obase(k), tbase(k);
    size_t o = 0;
    for (size_t j = 0; j < k; j++) {
        cfpq_ctx *c = qs[j]->ctx;
        c->last_stream = st;
        if (cudaMemcpyAsync(&s->h_state[j], c->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return CFPQ_ERR_CUDA;
        obase[j] = o;
        const int rc = count_all_enqueue(c, st, s->h_off + o);
        if (rc != CFPQ_OK) return rc;
        o += (size_t)c->n_nt + 1;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return CFPQ_ERR_CUDA;
    size_t total = 0;
    for (size_t j = 0; j < k; j++) {
        tbase[j] = total;
        total += (size_t)s->h_off[obase[j] + (size_t)qs[j]->ctx->n_nt];
    }
    // the triples' staging (page-locked); where it cannot grow, each query's triples go to
    // ordinary host memory one query at a time
    const bool staged = host_reserve(s->h_trip, s->trip_cap, total);
    for (size_t j = 0; j < k; j++) {
        Served *q = qs[j];
        cfpq_ctx *c = q->ctx;
        const int rc = apply_status(c, s->h_state[j]);
        q->status = rc;
        q->iterations = c->stats.iterations;
        c->solved = true;
        if (rc == CFPQ_ERR_CUDA) return rc;
        const size_t tj = (size_t)s->h_off[obase[j] + (size_t)c->n_nt];
        if (!staged) {
            const int r2 = extract_all_host(c, q->results);
            if (r2 != CFPQ_OK) return r2;
            continue;
        }
        if (tj == 0) continue;
        int r2 = ensure_triples(c, tj, st);
        if (r2 == CFPQ_OK) r2 = emit_all(c, c->d_triples, st);
        if (r2 != CFPQ_OK) return r2;
        if (cudaMemcpyAsync(s->h_trip + tbase[j], c->d_triples, tj * sizeof(cfpq_triple), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess)
            return CFPQ_ERR_CUDA;
    }
    if (staged && cudaStreamSynchronize(st) != cudaSuccess) return CFPQ_ERR_CUDA;
    for (size_t j = 0; j < k; j++) {
        Served *q = qs[j];
        cfpq_ctx *c = q->ctx;
        const unsigned long long *off = s->h_off + obase[j];
        if (staged) {
            const cfpq_triple *t = s->h_trip + tbase[j];
            q->results.assign(c->n_nt, {});
            for (int a = 0; a < c->n_nt; a++) q->results[a].assign(t + off[a], t + off[a + 1]);
        }
        ctx_destroy(c);
        q->ctx = nullptr;
        s->used -= q->footprint;
        q->state = (q->status == CFPQ_OK) ? CFPQ_QUERY_DONE : CFPQ_QUERY_FAILED;
        s->state_of[q->ticket] = q->state;
        s->finished[q->ticket] = q;
        s->just_finished.push_back(q->ticket);
        s->completed++;
    }
    return CFPQ_OK;
}

extern "C" int cfpq_server_step(cfpq_server *s, int32_t *n_completed) {
    if (!s) return CFPQ_ERR_INVALID;
    int done_now = 0;
    s->steps++;
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
    clk::time_point t_phase = clk::now();
    // 1) admission by free HBM, in arrival order
    while (!s->waiting.empty() && (int)(s->resident.size() + s->solo.size()) < s->max_resident) {
        Pending &p = s->waiting.front();
        if (p.footprint > s->budget) {
            Served *q = new Served();
            q->ticket = p.ticket;
            q->state = CFPQ_QUERY_FAILED;
            q->status = CFPQ_ERR_NOMEM;
            s->state_of[q->ticket] = q->state;
            s->finished[q->ticket] = q;
            s->just_finished.push_back(q->ticket);
            s->failed++;
            s->waiting.pop_front();
            done_now++;
            continue;
        }
        if (s->used + p.footprint > s->budget) break;
        cfpq_grammar_cnf g{p.n_nt, p.n_term, p.unary.data(), (int32_t)p.unary.size(), p.binary.data(),
                           (int32_t)p.binary.size(), p.eps.data(), (int32_t)p.eps.size()};
        cfpq_options o;
        cfpq_options_default(&o);
        o.path = CFPQ_PATH_GATHER;
        o.schedule = p.schedule;
        const bool solo = (p.n + 255u) / 256u * 256u >= kSoloRows;
        cfpq_ctx *c = nullptr;
        int rc = ctx_create_pooled(&g, p.n, p.edges.data(), p.edges.size(), o, solo ? s->solo_stream : s->stream, &c);
        if (rc == CFPQ_ERR_NOMEM) break;  // the pool could not serve it now: retry next step
        if (rc != CFPQ_OK) return rc;
        if (solo) {
            // seed and the single-query loop on the second stream, without waiting for them
            c->solved = false;
            c->last_stream = s->solo_stream;
            if (cudaEventRecord(c->ev0, s->solo_stream) != cudaSuccess ||
                (rc = enqueue_reset_and_seed(c, s->solo_stream)) != CFPQ_OK ||
                (rc = run_loop(c, s->solo_stream)) != CFPQ_OK || cudaEventRecord(c->ev1, s->solo_stream) != cudaSuccess) {
                ctx_destroy(c);
                return rc != CFPQ_OK ? rc : CFPQ_ERR_CUDA;
            }
            Served *q = new Served();
            q->ticket = p.ticket;
            q->ctx = c;
            q->solo = true;
            q->footprint = p.footprint;
            q->state = CFPQ_QUERY_RUNNING;
            s->state_of[q->ticket] = q->state;
            s->used += p.footprint;
            s->peak_used = std::max(s->peak_used, s->used);
            s->solo.push_back(q);
            s->waiting.pop_front();
            continue;
        }
        DevState st0;
        memset(&st0, 0, sizeof(st0));
        st0.max_iter = c->max_iter;
        if (cudaMemcpyAsync(c->d_state, &st0, sizeof(st0), cudaMemcpyHostToDevice, s->stream) != cudaSuccess) {
            ctx_destroy(c);
            return CFPQ_ERR_CUDA;
        }
        Served *q = new Served();
        q->ticket = p.ticket;
        q->ctx = c;
        q->footprint = p.footprint;
        q->state = CFPQ_QUERY_RUNNING;
        q->init = 1;
        s->state_of[q->ticket] = q->state;
        s->used += p.footprint;
        s->peak_used = std::max(s->peak_used, s->used);
        s->resident.push_back(q);
        s->waiting.pop_front();
    }
    // large queries whose single-query loop has finished
    auto retire_solo = [&]() -> int {
        std::vector<Served *> still, done;
        for (Served *q : s->solo) {
            const cudaError_t e = cudaEventQuery(q->ctx->ev1);
            if (e == cudaErrorNotReady) {
                still.push_back(q);
                continue;
            }
            if (e != cudaSuccess) return CFPQ_ERR_CUDA;
            done.push_back(q);
        }
        s->solo.swap(still);
        const int rc = retire_batch(s, done, s->solo_stream);
        if (rc != CFPQ_OK) {  // nothing was freed: the queries stay where they were
            s->solo.insert(s->solo.end(), done.begin(), done.end());
            return rc;
        }
        done_now += (int)done.size();
        return CFPQ_OK;
    };
    s->admit_ms += ms_since(t_phase);
    t_phase = clk::now();
    int src = retire_solo();
    s->retire_ms += ms_since(t_phase);
    if (src != CFPQ_OK) return src;
    if (s->resident.empty()) {
        if (n_completed) *n_completed = done_now;
        return CFPQ_OK;
    }
    // 2) one grouped launch over every resident query
    t_phase = clk::now();
    const int k = (int)s->resident.size();
    int rc = server_bufs(s, k);
    if (rc != CFPQ_OK) return rc;
    std::vector<BatchQuery> hb(k);
    std::vector<int> active(k, 1);
    bool any_jacobi = false;
    cfpq_batch_tuning tune;
    batch_tuning_snapshot(&tune);
    for (int j = 0; j < k; j++) {
        fill_batch_query(s->resident[j]->ctx, &hb[j], s->resident[j]->init, tune);
        // round budget: cheap queries run up to `rounds` executions per launch, expensive ones
        // fewer, so small queries are not held to the pace of a large one
        const double scale = 4096.0 / (double)s->resident[j]->ctx->n_pad;
        hb[j].max_rounds = std::max(1, std::min(s->rounds, (int)(s->rounds * scale * scale)));
        any_jacobi |= hb[j].q.schedule == CFPQ_SCHED_JACOBI;
    }
    rc = batch_buffers_upload(&s->bufs, hb.data(), active.data(), k, s->rounds, any_jacobi, s->stream);
    if (rc != CFPQ_OK) return rc;
    rc = batch_launch(s->bufs.ctl, s->bufs.bq, s->stream, tune.blocks_per_sm, nullptr);
    if (rc != CFPQ_OK) return rc;
    s->launches++;
    unsigned err = 0;
    if (cudaMemcpyAsync(active.data(), s->bufs.active, sizeof(int) * k, cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(&err, &s->bufs.ctl->error, sizeof(err), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return CFPQ_ERR_CUDA;
    if (err) return CFPQ_ERR_TIMEOUT;
    batch_record_profile(&s->bufs, s->stream);
    s->launch_ms += ms_since(t_phase);
    t_phase = clk::now();
    // 3) retire the queries that stopped
    std::vector<Served *> keep, stopped;
    for (int j = 0; j < k; j++) {
        Served *q = s->resident[j];
        q->init = 0;
        (active[j] ? keep : stopped).push_back(q);
    }
    s->resident.swap(keep);
    if ((rc = retire_batch(s, stopped, s->stream)) != CFPQ_OK) {  // nothing was freed
        s->resident.insert(s->resident.end(), stopped.begin(), stopped.end());
        return rc;
    }
    done_now += (int)stopped.size();
    rc = retire_solo();
    s->retire_ms += ms_since(t_phase);
    if (rc != CFPQ_OK) return rc;
    if (n_completed) *n_completed = done_now;
    return CFPQ_OK;
}

extern "C" int cfpq_server_completed(cfpq_server *s, int64_t *tickets, size_t cap, size_t *count) {
    if (!s || !count) return CFPQ_ERR_INVALID;
    *count = s->just_finished.size();
    if (!tickets) return CFPQ_OK;
    if (cap < s->just_finished.size()) return CFPQ_ERR_BUFFER;
    std::copy(s->just_finished.begin(), s->just_finished.end(), tickets);
    s->just_finished.clear();
    return CFPQ_OK;
}

extern "C" int cfpq_server_query_info(const cfpq_server *s, int64_t ticket, cfpq_query_info *out) {
    if (!s || !out) return CFPQ_ERR_INVALID;
    auto it = s->state_of.find(ticket);
    if (it == s->state_of.end()) return CFPQ_ERR_INVALID;
    memset(out, 0, sizeof(*out));
    out->state = it->second;
    auto f = s->finished.find(ticket);
    if (f != s->finished.end()) {
        out->status = f->second->status;
        out->iterations = f->second->iterations;
        out->n_nonterm = (int32_t)f->second->results.size();
    }
    return CFPQ_OK;
}

extern "C" int cfpq_server_result(const cfpq_server *s, int64_t ticket, int32_t A, cfpq_triple *buf, size_t cap,
                                  size_t *count) {
    if (!s || !count) return CFPQ_ERR_INVALID;
    auto f = s->finished.find(ticket);
    if (f == s->finished.end()) return s->state_of.count(ticket) ? CFPQ_ERR_NOT_SOLVED : CFPQ_ERR_INVALID;
    const Served *q = f->second;
    if (q->state != CFPQ_QUERY_DONE && q->results.empty()) return q->status ? q->status : CFPQ_ERR_NOT_SOLVED;
    if (A < 0 || A >= (int32_t)q->results.size()) return CFPQ_ERR_INVALID;
    const auto &r = q->results[A];
    *count = r.size();
    if (!buf) return CFPQ_OK;
    if (cap < r.size()) return CFPQ_ERR_BUFFER;
    if (!r.empty()) memcpy(buf, r.data(), r.size() * sizeof(cfpq_triple));
    return CFPQ_OK;
}

extern "C" int cfpq_server_release(cfpq_server *s, int64_t ticket) {
    if (!s) return CFPQ_ERR_INVALID;
    auto f = s->finished.find(ticket);
    if (f == s->finished.end()) return CFPQ_ERR_INVALID;
    delete f->second;
    s->finished.erase(f);
    s->state_of.erase(ticket);
    return CFPQ_OK;
}

extern "C" int cfpq_server_stats_get(const cfpq_server *s, cfpq_server_stats *out) {
    if (!s || !out) return CFPQ_ERR_INVALID;
    memset(out, 0, sizeof(*out));
    out->queued = (int64_t)s->waiting.size();
    out->resident = (int64_t)(s->resident.size() + s->solo.size());
    out->completed = s->completed;
    out->failed = s->failed;
    out->launches = s->launches;
    out->steps = s->steps;
    out->budget_bytes = s->budget;
    out->used_bytes = s->used;
    out->peak_used_bytes = s->peak_used;
    out->admit_ms = s->admit_ms;
    out->launch_ms = s->launch_ms;
    out->retire_ms = s->retire_ms;
    return CFPQ_OK;
}

extern "C" void cfpq_server_destroy(cfpq_server *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->solo_stream) cudaStreamSynchronize(s->solo_stream);
    for (Served *q : s->resident) {
        ctx_destroy(q->ctx);
        delete q;
    }
    for (Served *q : s->solo) {
        ctx_destroy(q->ctx);
        delete q;
    }
    for (auto &kv : s->finished) delete kv.second;
    if (s->bufs_cap) batch_buffers_free(&s->bufs);
    if (s->stream) {
        cudaStreamSynchronize(s->stream);
        cudaStreamDestroy(s->stream);
    }
    if (s->solo_stream) cudaStreamDestroy(s->solo_stream);
    if (s->h_state) cudaFreeHost(s->h_state);
    if (s->h_off) cudaFreeHost(s->h_off);
    if (s->h_trip) cudaFreeHost(s->h_trip);
    delete s;
}
