// Shared declarations of the batched (grouped persistent) closure.
#pragma once
#include "cfpq_internal.h"

namespace cfpq {

struct BatchQuery {
    QDesc q;                          // copy of the query's descriptor
    unsigned long long prod_items;    // warps of one product round: groups * n * chunks
    unsigned long long row_items;     // warps of one clear / merge pass: n_nt * n
    int cpl;                          // words per lane of the gather accumulator
    uint32_t nch;                     // column chunks per row
    int init;                         // 1: clear and seed this query at the start of the launch
    int max_rounds;                   // loop executions this query may run in this launch
};

struct BatchCtl {
    unsigned bar_count, bar_spare, error, n_active;   // bar_count: grid barrier (top bit flips per barrier)
    int k, max_rounds, any_jacobi, pad;
    unsigned long long limit_ns;      // whole-launch wall-clock limit (0 = none)
    unsigned long long start_ns;      // %globaltimer at launch start (set by the kernel)
    int *active;                      // [k] 1 while the query has not converged
    int *act;                         // [k] compacted active query ids of the current round
    unsigned long long *prod_off;     // [k+1] prefix sums of prod_items over act
    unsigned long long *row_off;      // [k+1] prefix sums of row_items over act
};

struct BatchBuffers {
    int k;
    BatchCtl *ctl;
    BatchQuery *bq;
    int *active, *act;
    unsigned long long *prod_off, *row_off;
};

int batch_buffers_alloc(BatchBuffers *b, int k);
int batch_buffers_upload(BatchBuffers *b, const BatchQuery *hb, const int *active, int k, int max_rounds,
                         bool any_jacobi, cudaStream_t s);
void batch_buffers_free(BatchBuffers *b);
int batch_launch(BatchCtl *d_ctl, const BatchQuery *d_bq, cudaStream_t s, int *grid_out);
void fill_batch_query(const cfpq_ctx *c, BatchQuery *b, int init);

}  // namespace cfpq
