/*
 * cfpq.h -- C ABI of the B300 (sm_103a) engine for relational-semantics context-free
 * path querying (CFPQ) by matrix transitive closure.
 *
 * The method (Azimov & Grigorev, "Context-Free Path Querying by Matrix
 * Multiplication"):
 *   - input: an edge-labelled directed graph D = (V, E), V = {0..n-1}, and a grammar
 *     G = (N, Sigma, P) whose productions are A -> B C and A -> x (Section 2); this ABI
 *     also accepts A -> eps, which adds the empty walk (m, m);
 *   - output: the context-free relations R_A = {(m, n) | some walk m -> n has a label
 *     string derived from A} for every A in N (Section 2), returned as (A, m, n) triples;
 *   - computation: Algorithm 1 (Section 4.2). One Boolean n x n matrix T_A is kept per
 *     non-terminal, seeded from the terminal edges (matrix initialisation), and
 *     T_A |= T_B x T_C over the Boolean semiring is applied for every production
 *     A -> B C until no bit changes (the closure a^cf, whose result is R_A by Theorem 2).
 *
 * Conventions for every entry point:
 *   - return value: CFPQ_OK (0) or one of the CFPQ_ERR_* codes below; no entry point
 *     aborts the process; cfpq_strerror() names a code;
 *   - the library copies every input array during the call; the caller keeps ownership
 *     of everything it passes and of every output buffer;
 *   - all device memory belongs to a context and is released by cfpq_destroy(); the
 *     contexts of cfpq_create take it from a memory pool of the library (one per device),
 *     which keeps what destroyed contexts released for the next ones until
 *     cfpq_trim_memory() hands it back to the system;
 *   - a context is not thread-safe; distinct contexts may be used from distinct threads.
 *
 * Limits: 1 <= n <= CFPQ_MAX_NODES, 1 <= |N| <= CFPQ_MAX_NONTERM.
 */
#ifndef CFPQ_H_
#define CFPQ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CFPQ_MAX_NODES 131072
#define CFPQ_MAX_NONTERM 64
#define CFPQ_NOALLOC_MAX_ROWS 65536   /* row limit of cfpq_extract_pairs_noalloc */

enum cfpq_status {
    CFPQ_OK = 0,
    CFPQ_ERR_INVALID = 1,     /* an id out of range, n out of range, NULL where data is required */
    CFPQ_ERR_NOMEM = 2,       /* device or host allocation failed (or admission refused) */
    CFPQ_ERR_NOT_SOLVED = 3,  /* results asked for before a successful cfpq_solve */
    CFPQ_ERR_ITER_LIMIT = 4,  /* the iteration cap was reached before the fixpoint */
    CFPQ_ERR_TIMEOUT = 5,     /* the wall-clock limit was reached before the fixpoint */
    CFPQ_ERR_CUDA = 6,        /* a CUDA runtime call failed (no device, launch error, ...) */
    CFPQ_ERR_BUFFER = 7,      /* output capacity smaller than the result */
    CFPQ_ERR_UNSUPPORTED = 8, /* option combination not available (e.g. tensor path on a non-sm_103 device) */
    CFPQ_ERR_NOT_FOUND = 9    /* the pair asked for is not in the relation */
};

/* A -> x : lhs is a non-terminal id in [0, n_nonterm), term a terminal id in [0, n_term). */
typedef struct { int32_t lhs, term; } cfpq_rule1;
/* A -> B C : all three are non-terminal ids. */
typedef struct { int32_t lhs, b, c; } cfpq_rule2;

/* A grammar in the normal form of Section 2 (plus A -> eps). Duplicate productions are
 * allowed and mean the same production (set semantics). */
typedef struct {
    int32_t n_nonterm, n_term;
    const cfpq_rule1 *unary;  int32_t n_unary;
    const cfpq_rule2 *binary; int32_t n_binary;
    const int32_t *eps_lhs;   int32_t n_eps;   /* non-terminals with A -> eps */
} cfpq_grammar_cnf;

/* Edge (src, label, dst) of E: src, dst in [0, n), label a terminal id. Multiple edges
 * between the same nodes add the union of their heads (Section 4.2, after Algorithm 1). */
typedef struct { uint32_t src; int32_t label; uint32_t dst; } cfpq_edge;

/* Result element: (A, m, n) with (m, n) in R_A. */
typedef struct { int32_t A; uint32_t m, n; } cfpq_triple;

enum cfpq_schedule {
    CFPQ_SCHED_INPLACE = 0,   /* products update T_A as soon as they finish (same least fixpoint) */
    CFPQ_SCHED_JACOBI = 1,    /* T_{k+1} = T_k u (T_k x T_k) exactly as Algorithm 1's loop body */
    CFPQ_SCHED_AUTO = 2       /* the library chooses: INPLACE in cfpq_solve; in batched solves and
                                 serving, the schedule the batch tuning holds for the query's size
                                 class (cfpq_batch_tuning). Every choice reaches the same least
                                 fixpoint; switching between loop executions keeps it exact */
};

enum cfpq_path {
    CFPQ_PATH_AUTO = 0,       /* per production group and loop execution, the cheaper of the two
                                 below, chosen on the device from the current pair counts (falls
                                 back to GATHER where tensor cores are not available); unless the
                                 schedule is JACOBI, 64 executions in a row that add at most 8
                                 pairs each end the loop and the WORKLIST path finishes the
                                 closure (cfpq_stats.iterations: the executions before that) */
    CFPQ_PATH_TENSOR = 1,     /* dense tcgen05 product of every production, every iteration */
    CFPQ_PATH_GATHER = 2,     /* CUDA-core bit-gather over changed bits only (semi-naive) */
    CFPQ_PATH_WORKLIST = 3    /* each new pair is joined with its partners (semi-naive at the grain
                                 of single pairs; warps of one block take batches of pairs, and
                                 periodic chains of single-successor steps run across many
                                 blocks): for long chains of tiny deltas; the loop count is not
                                 defined (reported as 1) */
};

/* Operand format of the tensor-core Boolean products (Section 2's product, one Boolean
 * matrix product per production). The 0/1 operands are unpacked from the bit-packed matrices
 * into a floating-point kind the tensor cores multiply exactly: every product of two ones is a
 * positive power of two and the F32 sum of non-negative terms is non-zero iff some AND is true,
 * so the thresholded accumulator is the Boolean OR of ANDs (counts stay far below 2^24). */
enum cfpq_tensor_kind {
    CFPQ_TENSOR_AUTO = 0,     /* FP4 */
    CFPQ_TENSOR_FP8 = 1,      /* E4M3 bytes, tcgen05 kind::f8f6f4 (K = 32 per instruction) */
    CFPQ_TENSOR_FP4 = 2       /* E2M1 nibbles, tcgen05 kind::mxf4 with unit UE8M0 scale factors
                                 (K = 64 per instruction): half the unpacked bytes and twice the
                                 MMA rate of FP8 */
};

typedef struct {
    int32_t schedule;         /* enum cfpq_schedule; default INPLACE */
    int32_t path;             /* enum cfpq_path; default AUTO */
    int32_t use_graph;        /* 1: fixpoint loop in a CUDA graph with a conditional while node
                                 and a device-side convergence flag (default); 0: host-driven loop */
    int32_t profile;          /* 1: host-driven loop that times every product launch with CUDA
                                 events (cfpq_stats.product_ms / product_launches); default 0 */
    int64_t max_iter;         /* iteration cap; 0 = |V|^2 |N| + 1 (Theorem 3's bound on changes) */
    double timeout_s;         /* wall-clock limit checked on the device; <= 0 = none */
    int32_t lengths;          /* 1: single-path semantics (Section 5) as well -- every pair also
                                 carries the length of one walk whose labels A derives; read it with
                                 cfpq_get_lengths, and the walk itself with cfpq_get_path. Needs
                                 schedule JACOBI (AUTO is taken as JACOBI), a matrix path (not
                                 WORKLIST) and fewer than 8192 distinct binary productions; adds
                                 two uint32 per (A, m, n) cell (a length and the derivation step
                                 that set it: 2 * n_pad^2 * |N| * 4 bytes) to the context. Default 0 */
    int32_t dense_tensor;     /* 0 (default): tensor-core products skip the K steps where either
                                 operand tile (128 x 128 bits of T_B, 256 x 128 bits of T_C^T) is
                                 all zero, and output tiles with no such step (occupancy bitmaps
                                 refreshed at the start of each loop execution for the operands
                                 that changed); 1: every K step of every tile, Algorithm 1's dense
                                 product as written. Both give the same result */
    int32_t tensor_kind;      /* enum cfpq_tensor_kind: operand format of the tensor-core products;
                                 default AUTO. Every kind gives the same result */
    uint32_t row_begin;       /* row block of a sharded solve (cfpq_block_*): the products of this
                                 context compute rows [row_begin, row_end) of every T_A. Both 0
                                 (default): every row, an ordinary context. Otherwise row_begin is
                                 a multiple of 256 and below row_end, and row_end is a multiple of
                                 256 or equal to n; needs schedule JACOBI (AUTO is taken as
                                 JACOBI), a matrix path (not WORKLIST) and no lengths */
    uint32_t row_end;
} cfpq_options;

typedef struct {
    int64_t iterations;       /* loop executions, the last being the one that changed nothing */
    int64_t new_bits;         /* pairs added by products (excludes the seed) */
    int64_t seed_bits;        /* pairs set by the matrix initialisation */
    int64_t tensor_products;  /* (production, iteration) pairs computed by the tensor path */
    int64_t gather_products;  /* (production, iteration) pairs computed by the gather path */
    double dense_ops;         /* 2 * n_pad^3 * tensor_products: Boolean ops the tensor path executed */
    double solve_ms;          /* device time of the last cfpq_solve (CUDA events) */
    uint32_t n_pad;           /* padded matrix side (multiple of 256) */
    int32_t status;           /* status of the last cfpq_solve */
    int64_t kernel_launches;  /* kernels the last cfpq_solve ran (a graph's body counted per execution) */
    int64_t product_launches; /* profile mode: product kernel launches timed */
    double product_ms;        /* profile mode: summed device time of those launches */
    double tensor_ms;         /* profile mode: the part of product_ms spent in tensor-core launches */
    int64_t tensor_launches;  /* profile mode: tensor-core product launches timed */
    double product_bytes;     /* profile mode: bytes the gather products read or wrote (rows
                                 scanned, rows gathered, result rows merged) */
    int64_t worklist_items;   /* worklist path: pairs joined with their partners */
    int32_t schedule;         /* schedule the last solve ran (INPLACE or JACOBI; AUTO resolved) */
    int32_t gather_cpl;       /* batched solves: gather tile width used (32-bit words per lane) */
    double useful_ops;        /* profile mode: 2 x sum over tensor products of sum_k nnz(column k
                                 of T_B) nnz(row k of T_C), the Boolean ops with both operands 1 */
    double lengths_ms;        /* lengths on, profile mode: summed device time of the length kernels */
    int64_t lengths_launches; /* lengths on, profile mode: length kernel launches timed */
    double lengths_splits;    /* lengths on, profile mode: (production, middle node k) splits the
                                 length kernels examined, i.e. sum over new pairs (A, i, j) and
                                 productions A -> B C of |{k : (i, k) in T_B, (k, j) in T_C}| */
    double tensor_live_ops;   /* Boolean ops the tensor-core products executed: 2 x 128 x 256 x 128
                                 per K step issued (equals dense_ops with dense_tensor = 1) */
    double worklist_setup_ms; /* worklist path: wall time of building its tables (CSR adjacency of
                                 the static relations, unique-successor and period power tables,
                                 all on the device), at cfpq_create or at the first hand-over;
                                 0 until then */
} cfpq_stats;

typedef struct cfpq_ctx cfpq_ctx;

/* Fills *opt with the defaults. Errors: INVALID if opt is NULL. */
int cfpq_options_default(cfpq_options *opt);

/*
 * Creates a context for one query -- the inputs of Algorithm 1 (Section 4.2): the
 * edge-labelled graph D = (V, E) with nodes 0 .. |V| - 1 and the grammar in normal form
 * (Section 2), and the matrix T of Algorithm 1 held as one Boolean n x n matrix per
 * non-terminal (Section 4.1: T_ij is a set of non-terminals; bit (i, j) of matrix A says
 * A in T_ij). Validates and copies the grammar and the edge list,
 * allocates the bit-packed matrices in device memory (row-major, n_pad = n rounded up to
 * a multiple of 256, bit j of row i in 32-bit word i * n_pad/32 + j/32 at bit j % 32),
 * and uploads the edges. Uses the current CUDA device.
 *   g       grammar; every id must be in range (INVALID otherwise)
 *   n       number of nodes, 1..CFPQ_MAX_NODES
 *   edges   host array of n_edges edges (may be NULL iff n_edges == 0)
 *   opt     options, NULL for defaults
 *   out     receives the context; untouched on error
 * Errors: INVALID, NOMEM, CUDA, UNSUPPORTED (tensor path unavailable; lengths with schedule
 * INPLACE or path WORKLIST).
 */
int cfpq_create(const cfpq_grammar_cnf *g, uint32_t n, const cfpq_edge *edges, size_t n_edges,
                const cfpq_options *opt, cfpq_ctx **out);

/*
 * Runs Algorithm 1 on the device: matrix initialisation from the edges, then the
 * closure loop until an iteration adds no pair. May be called again; each call starts
 * from the edges. Blocks until the fixpoint is reached (or a limit hits).
 *   stream  a cudaStream_t to run on, or NULL for the context's own stream
 * Errors: INVALID (NULL, or a row-block context of a sharded solve: see cfpq_block_start),
 * ITER_LIMIT, TIMEOUT, CUDA, UNSUPPORTED. After ITER_LIMIT or TIMEOUT the partial closure is
 * still readable with cfpq_get (it is a subset of the result).
 */
int cfpq_solve(cfpq_ctx *ctx, void *stream);

/*
 * The context-free relation R_A = {(m, n) : A in T_mn} read off the closure (Section 2's
 * definition; Theorem 2, Section 4.1: after the loop, A in T_mn iff there is a walk from
 * m to n whose labels A derives). Copies R_A as triples (A, m, n), sorted by (m, n), into
 * buf (host memory). With
 * buf == NULL only *count is set (the size query). Runs on the stream of the last
 * cfpq_solve. Errors: INVALID (A out of range, count NULL), NOT_SOLVED, BUFFER (cap <
 * count; *count still set), NOMEM, CUDA.
 */
int cfpq_get(cfpq_ctx *ctx, int32_t A, cfpq_triple *buf, size_t cap, size_t *count);

/* R_A as in cfpq_get (Theorem 2), but buf is device memory (cap triples) and nothing is
 * copied to the host except the count. Errors: as cfpq_get. */
int cfpq_get_device(cfpq_ctx *ctx, int32_t A, cfpq_triple *buf, size_t cap, size_t *count);

/* Every relation R_A of the closure at once (Theorem 2, Section 4.1; the worked example of
 * Section 4.3 lists all seven): triples (A, m, n) sorted by (A, m, n) into buf (host memory,
 * cap triples); buf == NULL: only *count. Errors: INVALID, NOT_SOLVED, BUFFER, NOMEM, CUDA. */
int cfpq_get_all(cfpq_ctx *ctx, cfpq_triple *buf, size_t cap, size_t *count);

/* Every R_A as in cfpq_get_all (Theorem 2), but buf is device memory (cap triples); one host
 * synchronisation (for the count) per call. buf == NULL: only *count. Errors: as cfpq_get_all. */
int cfpq_get_all_device(cfpq_ctx *ctx, cfpq_triple *buf, size_t cap, size_t *count);

/*
 * Single-path semantics (Section 5): R_A as in cfpq_get, triples sorted by (m, n) into buf,
 * and in lengths[t] the length l of the walk that triple t carries (host memory, cap
 * entries each; buf == NULL and lengths == NULL: only *count). The lengths follow the
 * paper's rule: an edge (m, x, n) gives every A -> x the length 1, A -> eps gives (m, m) the
 * length 0, and a loop execution that first derives (m, n) for A through A -> B C and a
 * middle node k gives it l_B(m, k) + l_C(k, n) from the matrices before that execution; a
 * length once set is kept. Where one execution derives (m, n) for A through several
 * productions or middle nodes, the paper does not say which length is kept: this library
 * keeps the smallest of them, so the result is unique. Every length is that of some walk
 * from m to n whose labels A derives; lengths of 2^32 - 1 or more read as UINT32_MAX.
 * Errors: INVALID (A out of range, count NULL, exactly one of buf and lengths NULL),
 * UNSUPPORTED (context created without options.lengths), NOT_SOLVED, BUFFER, NOMEM, CUDA.
 */
int cfpq_get_lengths(cfpq_ctx *ctx, int32_t A, cfpq_triple *buf, uint32_t *lengths, size_t cap, size_t *count);

/*
 * Single-path semantics (Section 5): one walk m = v_0 -x_1-> v_1 ... -x_l-> v_l = n whose
 * label string x_1 .. x_l the non-terminal A derives, of the length cfpq_get_lengths reports
 * for (A, m, n). The walk is rebuilt on the device from the derivation step each pair
 * recorded when its length was set (the production A -> B C and middle node k of the
 * smallest length, the smallest production index and then the smallest k among equal
 * lengths; an edge label for length 1, the smallest label where several edges qualify; the
 * empty walk for A -> eps), so no search is needed. nodes receives l + 1 node ids and labels
 * l terminal ids (host memory; cap = capacity of labels, nodes holds cap + 1). With nodes ==
 * NULL and labels == NULL only *len = l is set. The rebuild runs one device thread per walk,
 * one step per derivation node (about 2 l steps).
 * Errors: INVALID (A, m or n out of range, len NULL, exactly one of nodes and labels NULL),
 * UNSUPPORTED (context without options.lengths, or a length of UINT32_MAX), NOT_SOLVED,
 * NOT_FOUND ((m, n) not in R_A), BUFFER (cap < l; *len still set), NOMEM, CUDA.
 */
int cfpq_get_path(cfpq_ctx *ctx, int32_t A, uint32_t m, uint32_t n, uint32_t *nodes, int32_t *labels, size_t cap,
                  size_t *len);

/*
 * Sharded solve by row blocks. The paper's remark on parallelism (Section 7) is that the
 * matrix products of one loop execution may run on different GPUs independently. Here each
 * rank owns a block of rows: a context created with options.row_begin / row_end computes
 * rows [row_begin, row_end) of every product T_B x T_C, which needs those rows of T_B and all
 * of T_C, so every rank keeps all of T. After the products of an execution the ranks
 * exchange the new pairs of their rows, and every rank merges all of them (Algorithm 1's
 * loop body, Jacobi schedule: T_{k+1} = T_k u T_k x T_k). By induction every rank then holds
 * the same T_k after k executions, the loop stops on all ranks at the same execution, and
 * the result (read with cfpq_get and the other read-out calls) is the closure of Theorem 2.
 * The calls, in the order of one solve:
 *   cfpq_block_start     matrix initialisation from all edges (Algorithm 1, before the loop)
 *   then, per loop execution:
 *   cfpq_block_products  the products of the next execution, over the context's rows only
 *   cfpq_block_export    the new pairs of the context's rows as records, for the other ranks
 *   cfpq_block_import    (once per other rank) their records, ORed in as new pairs
 *   cfpq_block_finish    merge and end of the execution; *changed = 1 if the loop continues
 * until cfpq_block_finish reports *changed = 0. How the records travel between the ranks
 * (NCCL or any other transport) is the caller's; the library only packs and unpacks them.
 * A record is 2 + W 32-bit words: the non-terminal id, the row i, then the W = n_pad / 32
 * words of the row's new pairs (bit j of word j / 32 at bit j % 32); records come in no
 * particular order and importing is order-independent (an OR).
 * Each call runs on `stream` (NULL: the context's stream).
 */
/* Matrix initialisation of a sharded solve (every edge, all rows). Errors: INVALID (NULL,
 * or a context without a row block), CUDA. */
int cfpq_block_start(cfpq_ctx *ctx, void *stream);
/* The products of the next loop execution over the context's rows (asynchronous; nothing
 * is read back). Errors: INVALID, NOT_SOLVED (no cfpq_block_start since the last finished
 * solve), CUDA. */
int cfpq_block_products(cfpq_ctx *ctx, void *stream);
/* Packs the pairs that this execution's products added to the context's rows into buf
 * (device memory, cap_words 32-bit words) as records of 2 + W words and sets *words (host)
 * to the words written; returns after the packing is complete. At most (row_end -
 * row_begin) * n_nonterm records. Errors: INVALID, NOT_SOLVED, BUFFER (cap_words too small:
 * *words is the size needed, buf's contents undefined), CUDA. */
int cfpq_block_export(cfpq_ctx *ctx, uint32_t *buf, size_t cap_words, size_t *words, void *stream);
/* ORs another rank's records (device memory, words 32-bit words as cfpq_block_export wrote
 * them) into this execution's new pairs (asynchronous). Errors: INVALID (words not a
 * multiple of 2 + W, buf NULL with words > 0), NOT_SOLVED, CUDA; a record naming a
 * non-terminal or row out of range is skipped and makes cfpq_block_finish return INVALID. */
int cfpq_block_import(cfpq_ctx *ctx, const uint32_t *buf, size_t words, void *stream);
/* Merges this execution's new pairs (the context's own and the imported ones) into T and
 * ends the execution; *changed (host) = 1 if some rank added a pair, so the loop goes on,
 * 0 when the closure is complete (the context then counts as solved). Synchronises the
 * stream. Errors: INVALID (NULL, or an imported record out of range), NOT_SOLVED,
 * ITER_LIMIT, TIMEOUT, CUDA. */
int cfpq_block_finish(cfpq_ctx *ctx, void *stream, int32_t *changed);

/*
 * Checkpoint and resume of the fixpoint loop. After k executions of Algorithm 1's loop
 * (Section 4.2) the loop's whole state is T_k and the pairs the k-th execution added (the
 * next execution's semi-naive delta), with their row bitmaps and counts. The closure is
 * monotone with a unique least fixpoint (Theorem 2), so resuming from a saved state reaches
 * the same result as an uninterrupted solve, after the same total number of executions
 * under the Jacobi schedule. Only contexts on a matrix path without lengths, and not row
 * blocks, have this state (UNSUPPORTED otherwise).
 *   cfpq_state_size    bytes of a state image of this context (host memory)
 *   cfpq_export_state  copies the state after a cfpq_solve or cfpq_resume that returned
 *                      (OK, ITER_LIMIT or TIMEOUT) into buf (cap bytes); NOT_SOLVED before
 *                      any solve, UNSUPPORTED if the worklist path finished the solve, BUFFER
 *                      if cap is too small
 *   cfpq_import_state  loads an image into a context created with the same grammar, n and
 *                      edges (INVALID if the image does not fit it; the product path and the
 *                      schedule may differ, as every choice reaches the same fixpoint); a
 *                      cfpq_resume then continues the loop from it
 *   cfpq_resume        continues the loop of an interrupted solve (ITER_LIMIT, TIMEOUT) or
 *                      of an imported state without re-seeding: at most more_executions
 *                      further executions (0: up to Theorem 3's bound, |V|^2 |N| + 1
 *                      executions in all, whatever cap the context was created with), then as
 *                      cfpq_solve (the same statuses; the relations are read the same way).
 *                      NOT_SOLVED if there is nothing to resume
 * The image holds a header and then, bit-packed as on the device, T, the delta plane, its
 * row bitmap, T's row bitmap and T's word summary; it is tied to this library's layout.
 */
int cfpq_state_size(const cfpq_ctx *ctx, size_t *bytes);
int cfpq_export_state(cfpq_ctx *ctx, void *buf, size_t cap);
int cfpq_import_state(cfpq_ctx *ctx, const void *buf, size_t bytes);
int cfpq_resume(cfpq_ctx *ctx, void *stream, int64_t more_executions);

/* |R_A| without copying pairs (for the start symbol, the #results column of the tables of
 * Section 6, diagonal pairs included). Errors: as cfpq_get. */
int cfpq_count(cfpq_ctx *ctx, int32_t A, size_t *count);

/* Statistics of the last cfpq_solve: loop executions of Algorithm 1 (k of Section 4.3),
 * pairs added, Boolean products run and their dense work (Theorem 4's BMM terms), times.
 * Errors: INVALID. */
int cfpq_stats_get(const cfpq_ctx *ctx, cfpq_stats *out);

/* Releases the context and its device memory; NULL is ignored. Waits for the device's
 * outstanding work first (as cudaFree does), then returns the memory to the library's pool
 * of the context's device, where the next cfpq_create reuses it without a new allocation. */
void cfpq_destroy(cfpq_ctx *ctx);

/* Hands the device memory that the library's pool on the current device holds unused (what
 * destroyed contexts released) back to the system, keeping at most keep_bytes reserved
 * (0: everything unused). Memory of live contexts is not touched. Not part of the paper's
 * method: a memory-management call of this library. A pool that cannot allocate trims
 * itself this way once before it reports CFPQ_ERR_NOMEM. Errors: UNSUPPORTED (the device
 * has no memory pools), CUDA. */
int cfpq_trim_memory(size_t keep_bytes);

/* Static string naming a status code. */
const char *cfpq_strerror(int code);

/*
 * Reads grammar text into the normal form: one production per line, "A B C", "A x" or
 * "A eps", '#' starts a comment. A symbol is a non-terminal iff it is some line's
 * left-hand side; every other symbol must be one of the n_labels terminal names
 * (terminal id = position in labels). A terminal inside a binary production gets a
 * preterminal named "<x>" with the production <x> -> x, as the paper rewrites its
 * same-generation grammar into normal form (Section 4.3). Non-terminal ids: left-hand
 * sides in order of first appearance, then preterminals in order of first use.
 * On success *out owns its arrays; release it with cfpq_grammar_free.
 * Errors: INVALID (syntax, unknown terminal, chain production A -> B, too many
 * non-terminals); err (may be NULL, size errlen) receives a message.
 */
typedef struct cfpq_parsed_grammar cfpq_parsed_grammar;
int cfpq_grammar_parse(const char *text, const char *const *labels, int32_t n_labels,
                       cfpq_parsed_grammar **out, char *err, size_t errlen);
/* The normal form inside a parsed grammar (valid until cfpq_grammar_free). */
const cfpq_grammar_cnf *cfpq_grammar_cnf_of(const cfpq_parsed_grammar *pg);
/* Name of non-terminal id (NULL if out of range). */
const char *cfpq_grammar_name(const cfpq_parsed_grammar *pg, int32_t id);
void cfpq_grammar_free(cfpq_parsed_grammar *pg);

/*
 * Algorithm 1 (Section 4.2) for many independent queries at once. The paper solves one
 * query per call; grouping queries is this library's own, and each context still reaches
 * its own least fixpoint (Theorem 2, Section 4.1), the result of solving it alone.
 * Batched solve (many independent queries, one persistent grouped launch): every
 * context advances one loop iteration per round; a context whose iteration added no
 * pair is retired (per-query convergence) while the others continue. Results are
 * identical to solving each context alone. Each context keeps its own schedule and
 * iteration cap; products always take the gather path inside the grouped launch. The
 * smallest positive timeout_s among the contexts limits the whole launch (checked on the
 * device after every round; the contexts are then left unsolved). Contexts created with
 * options.lengths are not taken (UNSUPPORTED). Errors: INVALID, NOMEM,
 * CUDA, UNSUPPORTED (no cooperative launch; a lengths context), INVALID (also: a row-block
 * context), TIMEOUT (the launch's wall-clock limit passed
 * or a bounded grid barrier gave up), ITER_LIMIT (some context hit its cap; the others are
 * still complete).
 */
int cfpq_solve_batch(cfpq_ctx *const *ctxs, int32_t k, void *stream);

/*
 * Launch configuration of batched solves and serving steps, and its autotuner.
 *
 * The grouped launch spreads work items over a persistent grid; a product item is one row
 * i of one production group and a tile of 32 * cpl words of that row (one word per lane
 * per step, cpl words per lane), so cpl sets the tile shape: wide tiles scan the left
 * operand's row once for many output words, narrow tiles give more items for the same
 * row. Queries are put into size classes by their row length W = n_pad / 32 words: class
 * c holds 2^(c-1) < W <= 2^c (W >= 8, so the classes in use are 3 .. 21). Per class the
 * configuration gives cpl and the schedule taken by contexts created with
 * CFPQ_SCHED_AUTO; for the whole launch, the number of resident blocks per SM.
 *
 * Every configuration computes the same result (bit-identical triples); only the device
 * time and, for the schedule, the number of loop executions differ. A size class can also
 * leave the grouped launch (product = CFPQ_BATCH_ALONE): large, dense queries, whose own tiles
 * fill the GPU, then get tensor-core products, which the grouped launch does not run.
 */
#define CFPQ_TUNE_CLASSES 24
typedef struct {
    int32_t blocks_per_sm;                 /* 1 .. 8; 0 = the occupancy limit, at most 8 */
    int32_t cpl[CFPQ_TUNE_CLASSES];        /* 1, 2, 4 or 8; 0 = built-in (the smallest cpl with
                                              32 * cpl >= W, at most 8) */
    int32_t schedule[CFPQ_TUNE_CLASSES];   /* CFPQ_SCHED_INPLACE or _JACOBI for AUTO contexts */
    int32_t product[CFPQ_TUNE_CLASSES];    /* CFPQ_BATCH_GROUPED (0, built-in): the class's queries
                                              run in the grouped launch, whose products are gathers;
                                              CFPQ_BATCH_ALONE (1): they are solved beside it,
                                              concurrently, each by its own single-query loop on its
                                              context's stream, with the context's product path (the
                                              automatic path puts a product on the tensor cores,
                                              with tile skipping, where the cost model finds it
                                              cheaper). Same results either way */
} cfpq_batch_tuning;
#define CFPQ_BATCH_GROUPED 0
#define CFPQ_BATCH_ALONE 1

typedef struct {
    int32_t trials;        /* batched solves the tuner timed (the final confirmation included) */
    double default_ms;     /* device time of the batch with the built-in configuration */
    double best_ms;        /* device time with the configuration returned */
} cfpq_tune_report;

/* The built-in configuration (blocks_per_sm 0, cpl 0, schedule INPLACE). Host only. */
void cfpq_batch_tuning_default(cfpq_batch_tuning *t);
/* Copies the configuration batched solves and serving steps of this process use now. */
int cfpq_batch_tuning_get(cfpq_batch_tuning *t);
/* Installs a configuration after checking every field (INVALID if one is out of range;
 * nothing changes then). Host only; takes effect at the next batched launch. */
int cfpq_batch_tuning_set(const cfpq_batch_tuning *t);
/*
 * Autotuner: times batched solves of these contexts (each a complete solve from the seed,
 * so the contexts end solved, with the results of the last run) under candidate
 * configurations, by coordinate descent from the built-in one: blocks per SM (1, 2, 4, 8,
 * within occupancy), then cpl (1, 2, 4, 8) for each size class present, heaviest class
 * first, then the schedule of each class that holds AUTO contexts, then, for each class of
 * W > 32 words (heaviest first), solving its queries alone beside the launch. A candidate replaces
 * the current choice only if it is at least 3 % faster. Every step is timed with CUDA
 * events on `stream` (NULL: the first context's stream). The best configuration is
 * merged into the installed one (the classes present and blocks_per_sm), copied to
 * *best if best != NULL, and confirmed by one more run whose time is report->best_ms.
 * Errors: those of cfpq_solve_batch (nothing is installed then).
 */
int cfpq_autotune_batch(cfpq_ctx *const *ctxs, int32_t k, void *stream, cfpq_batch_tuning *best,
                        cfpq_tune_report *report);
/*
 * Measured throughput of the warp-level integer tensor instructions on this device, in
 * tera-ops/s (2 ops per multiply-add): mma.sync m16n8k32 s8 x s8 -> s32 and m16n8k256
 * b1 AND/popc -> s32. On sm_103a these are the only 8-bit integer and 1-bit tensor paths
 * (tcgen05 has no 8-bit integer kind there); the Boolean product's rate is also reported
 * against them. Runs two timed launches of a few tens of ms on the current device; not
 * part of any solve. Errors: INVALID (NULL output), NOMEM, CUDA.
 */
int cfpq_measure_mma_sync_peaks(double *s8_tops, double *b1_tops);

/*
 * Measured dense rate of the tcgen05 MMA kinds a Boolean product (Section 2's product
 * over subsets of N, one Boolean matrix product per production; the BMM term of Theorem 4)
 * can use on sm_103a, in the tile shape of the product kernels: M = 128, N = 256, A in
 * tensor memory, B in shared memory, F32 accumulation. One CTA per SM issues the MMAs back
 * to back with no unpacking, so these are the ceilings of the product kernels of each kind.
 * *_tflops: tera-ops/s over the device (2 ops per multiply-add, CUDA events around one
 * launch); *_ops_per_clk_sm: ops per SM clock cycle of one CTA (clock64 around its MMAs),
 * independent of the clock the device ran at; *_exact: 1 if every checked accumulator
 * element equals the exact sum of the known operands (all 1.0, unit scale factors), i.e.
 * the kind's operand encoding and instruction descriptor are the ones the kernels use.
 * Two timed launches of a few ms each on the current device; not part of any solve.
 * Errors: INVALID (NULL), UNSUPPORTED (not sm_103), NOMEM, CUDA.
 */
typedef struct {
    double f8f6f4_tflops;          /* kind::f8f6f4, E4M3 operands, K = 32 per instruction */
    double mxf4_tflops;            /* kind::mxf4 block-scaled, E2M1 operands, UE8M0 scales, K = 64 */
    double f8f6f4_ops_per_clk_sm;
    double mxf4_ops_per_clk_sm;
    int32_t f8f6f4_exact;
    int32_t mxf4_exact;
} cfpq_tensor_peaks;
int cfpq_measure_tensor_peaks(cfpq_tensor_peaks *out);

/* Batched solve under an explicit configuration instead of the installed one. */
int cfpq_solve_batch_tuned(cfpq_ctx *const *ctxs, int32_t k, const cfpq_batch_tuning *t, void *stream);
/*
 * Device time per phase of the last batched launch in this process (a batched solve or a
 * serving step), in ms summed over its rounds, and the number of rounds. Phases: 0 start
 * (clear, seed, first work tables), 1 scan (rows that take part in the products, and the
 * clear of the delta plane the products will write), 2 products, 3 Jacobi merge, 4
 * per-query end of iteration, 5 work-table rebuild; entries beyond 5 are set to 0. round_product_ms
 * (may be NULL when n_round_slots is 0) receives the products phase of each of the first
 * CFPQ_BATCH_PROFILE_ROUNDS rounds; other slots are set to 0. Host only.
 */
#define CFPQ_BATCH_PHASES 6
#define CFPQ_BATCH_PROFILE_ROUNDS 64
int cfpq_batch_last_profile(double *phase_ms, int32_t n_phases, int64_t *rounds, double *round_product_ms,
                            int32_t n_round_slots);

/*
 * Serving (continuous batching). A server takes independent queries (grammar + graph) at
 * any time, admits them in arrival order while their device footprint fits in an HBM
 * budget, and advances all resident queries together: each cfpq_server_step is one
 * persistent grouped launch that seeds the newly admitted queries and runs up to
 * rounds_per_step executions of Algorithm 1's loop body (Section 4.2) for every resident
 * query (fewer for large queries, so small ones are not held to their pace). A query whose loop stopped is retired: its R_A are copied to host memory and its
 * device memory is returned to a stream-ordered pool at once. Each query's result equals
 * solving it alone (its own least fixpoint).
 */
typedef struct cfpq_server cfpq_server;

enum cfpq_query_state { CFPQ_QUERY_QUEUED = 0, CFPQ_QUERY_RUNNING = 1, CFPQ_QUERY_DONE = 2, CFPQ_QUERY_FAILED = 3 };

typedef struct {
    uint64_t hbm_budget_bytes;  /* device bytes resident queries may hold; 0 = 90 % of free memory at creation */
    int32_t rounds_per_step;    /* most loop executions per step of a query (queries with n above
                                   4096 get proportionally fewer, at least one); 0 = 8 */
    int32_t max_resident;       /* upper bound on resident queries (at most 2^24); 0 = 4096 */
} cfpq_server_options;

typedef struct {
    int32_t state;              /* enum cfpq_query_state */
    int32_t status;             /* CFPQ_OK, NOMEM (larger than the whole budget), ITER_LIMIT, ... */
    int64_t iterations;         /* loop executions (when finished) */
    int32_t n_nonterm;          /* number of relations available (when finished) */
    int32_t reserved;
} cfpq_query_info;

typedef struct {
    int64_t queued, resident, completed, failed, launches, steps;
    uint64_t budget_bytes, used_bytes, peak_used_bytes;
    double admit_ms;   /* host wall time of the steps' admissions (context creation, uploads) */
    double launch_ms;  /* host wall time of the grouped launches, from issue to their results */
    double retire_ms;  /* host wall time of the retirements (status, every R_A to the host, free) */
} cfpq_server_stats;

/* Fills *opt with the defaults. Errors: INVALID. */
int cfpq_server_options_default(cfpq_server_options *opt);
/* Creates a server on the current device. Errors: INVALID, NOMEM, CUDA. */
int cfpq_server_create(const cfpq_server_options *opt, cfpq_server **out);
/* Queues a query (inputs copied; schedule = enum cfpq_schedule) and returns its ticket.
 * Nothing runs until cfpq_server_step. Errors: INVALID (as cfpq_create). */
int cfpq_server_submit(cfpq_server *s, const cfpq_grammar_cnf *g, uint32_t n, const cfpq_edge *edges,
                       size_t n_edges, int32_t schedule, int64_t *ticket);
/* Admission, one grouped launch, retirement; *n_completed (may be NULL) receives the number
 * of queries that finished or failed in this step. Errors: CUDA, TIMEOUT (a bounded device
 * wait gave up). */
int cfpq_server_step(cfpq_server *s, int32_t *n_completed);
/* Tickets that finished or failed since the previous call (then forgotten by this list);
 * tickets == NULL: only *count. Errors: INVALID, BUFFER (cap < count). */
int cfpq_server_completed(cfpq_server *s, int64_t *tickets, size_t cap, size_t *count);
/* State of a ticket. Errors: INVALID (unknown or released ticket). */
int cfpq_server_query_info(const cfpq_server *s, int64_t ticket, cfpq_query_info *out);
/* R_A of a finished query as triples sorted by (m, n), host memory, two-call size query.
 * Errors: INVALID, NOT_SOLVED (still queued or running), BUFFER, the query's own failure status. */
int cfpq_server_result(const cfpq_server *s, int64_t ticket, int32_t A, cfpq_triple *buf, size_t cap,
                       size_t *count);
/* Forgets a finished query's host results. Errors: INVALID (unknown or unfinished ticket). */
int cfpq_server_release(cfpq_server *s, int64_t ticket);
/* Counters of the server. Errors: INVALID. */
int cfpq_server_stats_get(const cfpq_server *s, cfpq_server_stats *out);
/* Waits for the server's device work, frees everything; NULL is ignored. */
void cfpq_server_destroy(cfpq_server *s);

/*
 * Allocation-free pair extraction (the paper has no counterpart; it is an interface for
 * callers that cannot allocate device memory, e.g. code under an external allocator that
 * owns the device heap, or paths where cudaMalloc is forbidden after start-up).
 * Reads a bit-packed relation matrix that the caller owns in device memory -- n_rows rows
 * of row_words 32-bit words, bit j of row i at word i * row_words + j / 32, bit j % 32
 * (the layout of the engine's matrices) -- and writes its pairs (m, n), n < n_cols, as
 * triples (A, m, n) sorted by (m, n) into the caller's device buffer out (cap triples).
 * With out == NULL only *count (host) is set. Runs on `stream` (NULL = legacy default
 * stream) and returns after the work is complete.
 * The library allocates nothing for this call: its scratch is one fixed device array
 * that every GPU loading the library holds until the process exits (~768 KiB). The
 * first call on a device (and again in a new CUDA context of that device, e.g. after a
 * device reset) looks up that array's device address with the device current. All calls
 * share the array: calls whose work overlaps on the GPU race and must be serialised by the
 * caller. Every call synchronises `stream` and reads the pair count on the host, so it
 * must never be made on a stream that is being captured into a CUDA graph: such a call is
 * refused (INVALID) before any device work, and the capture stays intact.
 * Errors: INVALID (count NULL, bits NULL with n_rows > 0, n_rows > CFPQ_NOALLOC_MAX_ROWS,
 * n_cols > 32 * row_words, stream capturing), BUFFER (cap < count; *count still set), CUDA.
 */
int cfpq_extract_pairs_noalloc(const uint32_t *bits, uint32_t n_rows, uint32_t n_cols, uint32_t row_words,
                               int32_t A, cfpq_triple *out, size_t cap, size_t *count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CFPQ_H_ */
