// Host-side context of one query and the declarations shared by the engine's files.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cfpq.h"
#include "cfpq_device.cuh"

struct cfpq_ctx {
    // problem
    uint32_t n = 0, n_pad = 0, W = 0;
    uint64_t plane = 0;
    int n_nt = 0, n_term = 0, n_groups = 0, n_unary = 0, n_eps_rules = 0;
    size_t n_edges = 0;
    int schedule = 0, path = 0, use_graph = 1, profile = 0;
    int schedule_req = 0;          // as requested (CFPQ_SCHED_AUTO resolved per launch kind)
    double timeout_s = 0.0;
    uint64_t max_iter = 0;
    std::vector<cfpq::Rule> rules;
    std::vector<int32_t> gstart;
    std::vector<char> group_tensor;   // per group: 1 = tensor-core product
    std::vector<char> nt_dynamic;     // per non-terminal: 1 = left-hand side of a binary production
    bool auto_mixed = false;          // AUTO path with tensor cores: product kind chosen per group and iteration
    bool any_gather = false;          // some group may take the gather product
    bool allow_switch = false;        // AUTO, not Jacobi: a long run of tiny deltas hands over to the worklist
    bool switched = false;            // the last solve finished on the worklist path
    uint32_t *d_list = nullptr;       // gather items of one loop execution (in the arena)
    uint32_t *d_colcnt = nullptr;     // profile mode: column counts of a left operand (n_pad)
    uint32_t list_cap = 0;
    bool lengths = false;             // single-path semantics: a length plane per non-terminal
    uint32_t *d_L = nullptr;          // [n_nt][n_pad][n_pad] lengths (in the arena)
    uint32_t *d_Wit = nullptr;        // [n_nt][n_pad][n_pad] derivation step of each pair (in the arena)
    uint64_t lplane = 0;              // cells per length plane = n_pad * n_pad
    uint32_t *d_occA = nullptr, *d_occB = nullptr;  // tile occupancy (tensor path with tile skipping; arena)
    uint32_t *d_occCA = nullptr, *d_occCB = nullptr, *d_occKnown = nullptr;  // its counts per K slice (arena)
    void *d_tile_list = nullptr;      // tile skipping: live output tiles of one product (uint2 each; arena)
    bool dense_tensor = false;        // tensor products over every K step (no tile skipping)
    int tensor_kind = CFPQ_TENSOR_FP4;  // operand format of the tensor products (FP8 or FP4, resolved)
    bool resumable = false;           // the device holds an interrupted or imported loop state (cfpq_resume)
    bool block = false;               // sharded solve: the products compute rows [row0, row1) only
    bool block_started = false;       // cfpq_block_start ran and the solve has not finished yet
    uint32_t row0 = 0, row1 = 0;      // the row block (row1 = n_pad for the last block)
    uint32_t *d_Tsum = nullptr;       // word summary of T (in the arena)
    uint32_t *d_TTsum = nullptr;      // word summary of T^T (lengths only; in the arena)
    uint32_t SW = 0;                  // summary words per row: ceil(W / 32) rounded up to a multiple of 4
    int len_grid = 0;                 // persistent grid of the length kernel
    uint32_t *d_lens = nullptr;       // extraction: lengths of the emitted triples
    size_t lens_cap = 0;
    int gather_grid = 0;              // persistent grid of the listed gathers
    int loop_grid = 0;                // cooperative grid of the persistent gather loop (0: not used)
    int sms = 148;                    // multiprocessors of the device (grid-stride kernels use a few blocks per SM)
    // device memory
    uint32_t *d_T = nullptr, *d_TT = nullptr, *d_X0 = nullptr, *d_X1 = nullptr;
    uint32_t *d_R0 = nullptr, *d_R1 = nullptr, *d_Trow = nullptr;
    cfpq::Rule *d_rules = nullptr;
    int32_t *d_gstart = nullptr;
    int2 *d_nt_rules = nullptr;       // per non-terminal: range of its productions in d_rules
    int2 *d_unary = nullptr;
    int32_t *d_eps = nullptr;
    cfpq_edge *d_edges = nullptr;
    cfpq::DevState *d_state = nullptr;
    cfpq::DevState *d_state0 = nullptr;      // the loop state every solve starts from (fixed at create)
    cfpq::QDesc *d_q = nullptr;
    cfpq::QDesc hq{};
    void *d_arena = nullptr;                 // every buffer below lives in this one allocation
    uint32_t *d_counts = nullptr;            // [n_nt * n_pad] pairs per (non-terminal, row)
    uint64_t *d_offsets = nullptr;           // [n_nt * n_pad] exclusive prefix of d_counts
    unsigned long long *d_block_sums = nullptr;
    unsigned long long *d_nt_off = nullptr;  // [n_nt + 1] first triple of each non-terminal
    unsigned long long *d_total = nullptr;
    cfpq_triple *d_triples = nullptr;
    size_t triples_cap = 0;
    void *d_tc_work = nullptr;
    uint8_t *d_TTn = nullptr;                // E2M1 products: T^T as nibbles (n_nt x n_pad rows of n_pad / 2 bytes)
    void *h_tc_work = nullptr;               // tensor path: tensor maps (host side)
    void *h_wl = nullptr;                    // worklist path state
    std::vector<int2> h_unary;               // (lhs, terminal) productions, host copy
    std::vector<int32_t> h_eps;
    std::vector<int2> h_nt_rules;            // host copy of d_nt_rules (kept alive for the async copy)
    // execution
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool pooled = false;                     // a server's context: runs on the server's stream
    cudaMemPool_t pool = nullptr;            // every device buffer of the context comes from this pool
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t aux_stream = nullptr;       // capture the branches of the AUTO choice nodes
    cudaStream_t aux2_stream = nullptr;
    std::vector<cudaGraphConditionalHandle> h_choice;  // per group: IF (tensor) / ELSE (gather); then "any tensor"
    cudaGraphConditionalHandle *d_choice = nullptr;    // device copy of h_choice (in the arena)
    cudaStream_t last_stream = nullptr;      // stream of the last cfpq_solve (results are read on it)
    int64_t iter_launches = 0;               // kernels one loop execution launches
    int64_t fixed_launches = 0;              // kernels a solve launches outside the loop
    std::vector<cudaEvent_t> prof_ev;        // profile mode: a start/stop pair per group
    bool solved = false;
    bool clean = false;                      // after a solve that converged on the matrix path: X0, X1
                                             // are zero and T is zero outside the rows Trow flags
    cfpq_stats stats{};
};

namespace cfpq {

constexpr int kScanSeg = 8192;                                  // cells per block of the wide scan
constexpr int kScanMaxBlocks = (CFPQ_MAX_NONTERM * CFPQ_MAX_NODES) / kScanSeg;

int ctx_init(cfpq_ctx *c, const cfpq_grammar_cnf *g, uint32_t n, const cfpq_edge *edges, size_t n_edges,
             const cfpq_options &o);
int validate_inputs(const cfpq_grammar_cnf *g, uint32_t n, const cfpq_edge *edges, size_t n_edges,
                    const cfpq_options *opt);
// Creates a context whose device memory comes from the device's default memory pool and
// which runs on `pool_stream` (used by the server); inputs must be validated already.
int ctx_create_pooled(const cfpq_grammar_cnf *g, uint32_t n, const cfpq_edge *edges, size_t n_edges,
                      const cfpq_options &o, cudaStream_t pool_stream, cfpq_ctx **out);
void ctx_destroy(cfpq_ctx *c);
// The library's memory pool on device `dev`: the contexts of cfpq_create allocate from it,
// and memory they free stays reserved in it for the next context (cfpq_trim_memory returns
// it to the system). Created on first use; nullptr if the device has no memory pools.
cudaMemPool_t library_pool(int dev);
// Stream-ordered allocation of `bytes` from the context's pool on stream s; when the pool is
// out of memory it gives back what it holds unused and tries once more.
cudaError_t ctx_alloc(cfpq_ctx *c, void **p, size_t bytes, cudaStream_t s);
void ctx_free(cfpq_ctx *c, void *p, cudaStream_t s);
int ensure_triples(cfpq_ctx *c, size_t total, cudaStream_t s);
int count_all_enqueue(cfpq_ctx *c, cudaStream_t s, unsigned long long *h_nt_off);
int emit_all(cfpq_ctx *c, cfpq_triple *out, cudaStream_t s);
int extract_all_host(cfpq_ctx *c, std::vector<std::vector<cfpq_triple>> &out);
// Bytes of device memory a context for this query holds (path GATHER unless tensor).
size_t query_footprint(uint32_t n, int n_nt, size_t n_edges, int n_rules, bool tensor);
void free_ctx_device(cfpq_ctx *c);
int enqueue_reset_and_seed(cfpq_ctx *c, cudaStream_t s);
int enqueue_iteration(cfpq_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h, int use_handle);
void arm_deadline(cfpq_ctx *c, cudaStream_t s);
// Copies the device state, applies it to the statistics; *to_worklist (may be NULL) receives
// whether the loop stopped to hand over to the worklist path.
int read_status(cfpq_ctx *c, cudaStream_t s, unsigned *to_worklist = nullptr);
int enqueue_tensor_transposes_gated(cfpq_ctx *c, int g, cudaStream_t s);
int enqueue_useful_work(cfpq_ctx *c, int g, cudaStream_t s);
int tensor_prepare(cfpq_ctx *c);
int enqueue_all_transposes(cfpq_ctx *c, cudaStream_t s);
int enqueue_transpose_bits(cfpq_ctx *c, int a, cudaStream_t s);  // TT[a] = T[a]^T, bit-packed
// Statistics and status of a solve from a copy of its device state.
int apply_status(cfpq_ctx *c, const DevState &st);
int run_loop(cfpq_ctx *c, cudaStream_t s);
// cfpq_solve in two parts: solve_begin enqueues the solve on s (no host synchronisation),
// solve_end waits for it and finishes it (status, worklist hand-over, statistics).
int solve_begin(cfpq_ctx *c, cudaStream_t s);
int solve_end(cfpq_ctx *c, cudaStream_t s);
uint32_t gather_chunks(uint32_t W, int *cpl);

// tensor-core product path (cfpq_tensor.cu)
bool tensor_path_available();
int enqueue_tensor_transposes(cfpq_ctx *c, int g, cudaStream_t s);
int enqueue_tensor_group(cfpq_ctx *c, int g, cudaStream_t s);
int enqueue_tensor_occupancy(cfpq_ctx *c, cudaStream_t s);
constexpr double kTcOpsPerStep = 2.0 * 128 * 256 * 128;  // Boolean ops of one K step of a tensor tile
int enqueue_tensor_seed_transposes(cfpq_ctx *c, cudaStream_t s, int64_t *launches);
void tensor_release(cfpq_ctx *c);

// single-path lengths (cfpq_lengths.cu)
int lengths_enqueue_seed(cfpq_ctx *c, cudaStream_t s);
int lengths_enqueue_iteration(cfpq_ctx *c, cudaStream_t s);
int lengths_of_triples(cfpq_ctx *c, const cfpq_triple *d_tr, size_t count, uint32_t *d_out, cudaStream_t s);
int lengths_rules_ok(const cfpq_ctx *c);  // few enough productions for the derivation-step encoding
int lengths_path(cfpq_ctx *c, int32_t A, uint32_t m, uint32_t n, uint32_t len, uint32_t *nodes, int32_t *labels);

// worklist path (cfpq_worklist.cu)
// seeded: T holds the seed already (a hand-over from the matrix loop); else it is seeded here
int worklist_setup(cfpq_ctx *c, bool seeded);
// from_delta: continue a closure the matrix loop started (stack = the current delta pairs,
// T^T rebuilt from T); otherwise a full solve from the seeds.
int worklist_run(cfpq_ctx *c, cudaStream_t s, bool from_delta = false);
void worklist_release(cfpq_ctx *c);

}  // namespace cfpq
