// Shared declarations of the batched (grouped persistent) closure.
#pragma once
#include "cfpq_internal.h"

namespace cfpq {

constexpr int kBatchPhases = 6;
constexpr int kMaxBatch = 1 << 24;  // queries per launch (product items carry a 24-bit index)
constexpr int kProfRounds = CFPQ_BATCH_PROFILE_ROUNDS;

struct BatchQuery {
    QDesc q;                          // copy of the query's descriptor
    unsigned long long prod_items;    // candidate-scan items of one round: groups * row words
    unsigned long long row_slots;     // most (group, row, chunk) product items one round can list
    unsigned long long row_items;     // warps of one clear / merge pass: n_nt * n
    int cpl;                          // words per lane of the gather accumulator
    uint32_t nch;                     // column chunks per row
    int init;                         // 1: clear and seed this query at the start of the launch
    int max_rounds;                   // loop executions this query may run in this launch
    unsigned long long max_iter;      // the query's iteration cap (set into its state at init)
    // start-of-launch work of init queries, flattened over the batch (host prefix sums):
    // clear chunks of [T, X1 end) and [R0, Trow end), then seed chunks of edges and eps pairs
    uint4 *clr_a, *clr_b;
    unsigned long long clr_a_n, clr_b_n;   // uint4 counts
    unsigned long long clr_off, seed_off;  // first chunk of this query in each phase
};

struct BatchCtl {
    unsigned bar_count, bar_spare, error, n_active;   // bar_count: grid barrier (top bit flips per barrier)
    int k, max_rounds, any_jacobi, pad;
    unsigned long long clr_total, seed_total;  // chunks of the two start phases
    unsigned long long *list;         // product items of the current round (packed, see pack_item)
    unsigned long long list_cap, list_len;
    unsigned long long limit_ns;      // whole-launch wall-clock limit (0 = none)
    unsigned long long start_ns;      // %globaltimer at launch start (set by the kernel)
    int *active;                      // [k] 1 while the query has not converged
    int *act;                         // [k] compacted active query ids of the current round
    unsigned long long *prod_off;     // [k+1] prefix sums of prod_items over act
    unsigned long long *row_off;      // [k+1] prefix sums of row_items over act
    // device time per phase, summed over rounds (block 0 reads %globaltimer after each
    // barrier): 0 start (clear, seed, first tables), 1 scan (candidate rows, clear of the
    // previous delta), 2 products, 3 Jacobi merge, 4 per-query tails, 5 table rebuild;
    // and the rounds run
    unsigned long long phase_ns[kBatchPhases];
    unsigned long long rounds;
    unsigned long long round_product_ns[kProfRounds];  // products phase of rounds 0 .. kProfRounds-1
};

struct BatchBuffers {
    int k;
    BatchCtl *ctl;
    BatchQuery *bq;
    int *active, *act;
    unsigned long long *prod_off, *row_off;
    DevState *states;                 // [k] copies of the queries' states after a launch
    unsigned long long *list;         // product item list, list_cap entries
    unsigned long long list_cap;
};

int batch_buffers_alloc(BatchBuffers *b, int k);
// Records the phase times and round count of the launch that used b (after it finished).
void batch_record_profile(const BatchBuffers *b, cudaStream_t s);
// Copies the k queries' device states into b->states (one small launch).
int batch_collect_states(const BatchBuffers *b, const BatchQuery *d_bq, int k, cudaStream_t s);
// Computes the start-phase prefix sums in hb, then copies control block and descriptors.
// limit_ns: wall-clock limit of the launch, checked after every round (0 = the default cap).
int batch_buffers_upload(BatchBuffers *b, BatchQuery *hb, const int *active, int k, int max_rounds,
                         bool any_jacobi, cudaStream_t s, unsigned long long limit_ns = 0);
void batch_buffers_free(BatchBuffers *b);
int batch_launch(BatchCtl *d_ctl, const BatchQuery *d_bq, cudaStream_t s, int blocks_per_sm, int *grid_out);
// Descriptor of one query for a grouped launch under configuration t: tile width (cpl) and,
// for CFPQ_SCHED_AUTO contexts, the schedule of the query's size class.
void fill_batch_query(const cfpq_ctx *c, BatchQuery *b, int init, const cfpq_batch_tuning &t);
void batch_tuning_snapshot(cfpq_batch_tuning *t);  // the installed configuration
int batch_size_class(uint32_t W);

}  // namespace cfpq
