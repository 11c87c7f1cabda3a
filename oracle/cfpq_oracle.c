/*
 * CPU oracle for relational-semantics context-free path querying.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or call this
 * file: only the test-suite, the smoke check and the benchmark's CPU-baseline leg do.
 *
 * What it computes (Section 2, the definition of the context-free relations R_A, and
 * Theorem 2 of Section 4.1, which states that the matrix closure reaches exactly
 * these relations): the least set of triples (A, m, n) closed under
 *     (A, m, n)  if (m, x, n) is an edge and A -> x is a production        (seed)
 *     (A, m, m)  if A -> eps is a production                                 (empty walk)
 *     (A, m, k)  if (B, m, n) and (C, n, k) and A -> B C is a production     (join)
 * computed with a worklist in the style of Hellings' algorithm for the relational
 * semantics (the algorithm the paper cites in Section 3): every derived triple is
 * inserted once and, when it is popped, joined against all triples already known on
 * either side. No blocking, no reordering of rules, no matrix products.
 *
 * Data structures: for each non-terminal A and node v, an out-set Out_A[v] (bit j set
 * iff (A, v, j) known) and an in-set In_A[v] (bit i set iff (A, i, v) known), both as
 * plain 64-bit-word bitsets. The scan "all k with (C, n, k) known and (A, m, k) not yet
 * known" is the word-wise Out_C[n] & ~Out_A[m].
 *
 * Building with -DORACLE_PLANT=<k> compiles a deliberately wrong variant (used only by
 * the tests that check the pins are sensitive): 1 drops the right-operand join, 2
 * ignores eps productions, 3 joins with the operands swapped (A -> C B).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

typedef struct {
    int32_t n_nt;
    int32_t n;
    int64_t words;      /* 64-bit words per bitset row */
    uint64_t *out;      /* [n_nt][n][words] */
    uint64_t *in;       /* [n_nt][n][words] */
    int64_t *count;     /* [n_nt] */
    int64_t total;
    int64_t pops;
} oracle_result;

typedef struct {
    uint32_t *v;        /* triples (A, m, n) */
    int64_t len, cap;
} stack_t_;

static int push(stack_t_ *s, uint32_t a, uint32_t m, uint32_t n) {
    if (s->len == s->cap) {
        int64_t nc = s->cap ? s->cap * 2 : 1 << 16;
        uint32_t *nv = (uint32_t *)realloc(s->v, (size_t)nc * 3 * sizeof(uint32_t));
        if (!nv) return -1;
        s->v = nv;
        s->cap = nc;
    }
    s->v[3 * s->len + 0] = a;
    s->v[3 * s->len + 1] = m;
    s->v[3 * s->len + 2] = n;
    s->len++;
    return 0;
}

static inline uint64_t *row(uint64_t *base, const oracle_result *r, int32_t a, int64_t v) {
    return base + ((int64_t)a * r->n + v) * r->words;
}

/* insert (a, m, n); returns 1 if new, 0 if known, -1 on allocation failure */
static int add(oracle_result *r, stack_t_ *w, int32_t a, int64_t m, int64_t n) {
    uint64_t *o = row(r->out, r, a, m);
    uint64_t bit = 1ull << (n & 63);
    if (o[n >> 6] & bit) return 0;
    o[n >> 6] |= bit;
    row(r->in, r, a, n)[m >> 6] |= 1ull << (m & 63);
    r->count[a]++;
    r->total++;
    return push(w, (uint32_t)a, (uint32_t)m, (uint32_t)n) ? -1 : 1;
}

void oracle_release(oracle_result *r) {
    if (!r) return;
    free(r->out);
    free(r->in);
    free(r->count);
    free(r);
}

/*
 * unary:  n_unary pairs (lhs, terminal)
 * binary: n_binary triples (lhs, left, right)
 * eps:    n_eps non-terminal ids with an A -> eps production
 * edges:  n_edges triples (src, label, dst)
 * Returns NULL on invalid input (ids out of range) or allocation failure.
 */
oracle_result *oracle_solve(int32_t n_nt, int32_t n_terms, int32_t n,
                            const int32_t *unary, int32_t n_unary,
                            const int32_t *binary, int32_t n_binary,
                            const int32_t *eps, int32_t n_eps,
                            const int64_t *edges, int64_t n_edges) {
    if (n_nt <= 0 || n < 0 || n_terms < 0) return NULL;
    for (int32_t i = 0; i < n_unary; i++)
        if (unary[2 * i] < 0 || unary[2 * i] >= n_nt || unary[2 * i + 1] < 0 || unary[2 * i + 1] >= n_terms)
            return NULL;
    for (int32_t i = 0; i < 3 * n_binary; i++)
        if (binary[i] < 0 || binary[i] >= n_nt) return NULL;
    for (int32_t i = 0; i < n_eps; i++)
        if (eps[i] < 0 || eps[i] >= n_nt) return NULL;
    for (int64_t e = 0; e < n_edges; e++)
        if (edges[3 * e] < 0 || edges[3 * e] >= n || edges[3 * e + 2] < 0 || edges[3 * e + 2] >= n ||
            edges[3 * e + 1] < 0 || edges[3 * e + 1] >= n_terms)
            return NULL;

    oracle_result *r = (oracle_result *)calloc(1, sizeof(oracle_result));
    if (!r) return NULL;
    r->n_nt = n_nt;
    r->n = n;
    r->words = (n + 63) / 64;
    size_t cells = (size_t)n_nt * (size_t)n * (size_t)r->words;
    r->out = (uint64_t *)calloc(cells ? cells : 1, sizeof(uint64_t));
    r->in = (uint64_t *)calloc(cells ? cells : 1, sizeof(uint64_t));
    r->count = (int64_t *)calloc((size_t)n_nt, sizeof(int64_t));
    stack_t_ w = {0, 0, 0};
    if (!r->out || !r->in || !r->count) goto fail;

    /* seeds: terminal edges */
    for (int64_t e = 0; e < n_edges; e++) {
        int64_t src = edges[3 * e], lab = edges[3 * e + 1], dst = edges[3 * e + 2];
        for (int32_t u = 0; u < n_unary; u++)
            if (unary[2 * u + 1] == lab && add(r, &w, unary[2 * u], src, dst) < 0) goto fail;
    }
    /* seeds: empty walks */
#if ORACLE_PLANT != 2
    for (int32_t i = 0; i < n_eps; i++)
        for (int64_t m = 0; m < n; m++)
            if (add(r, &w, eps[i], m, m) < 0) goto fail;
#endif

    while (w.len > 0) {
        w.len--;
        int32_t b = (int32_t)w.v[3 * w.len];
        int64_t m = w.v[3 * w.len + 1], nn = w.v[3 * w.len + 2];
        r->pops++;
        for (int32_t p = 0; p < n_binary; p++) {
            int32_t a = binary[3 * p], left = binary[3 * p + 1], right = binary[3 * p + 2];
#if ORACLE_PLANT == 3
            { int32_t t = left; left = right; right = t; }
#endif
            if (left == b) {
                /* (b, m, nn) as left operand: all k with (right, nn, k) known */
                const uint64_t *oc = row(r->out, r, right, nn);
                const uint64_t *oa = row(r->out, r, a, m);
                for (int64_t wd = 0; wd < r->words; wd++) {
                    uint64_t cand = oc[wd] & ~oa[wd];
                    while (cand) {
                        int64_t k = wd * 64 + __builtin_ctzll(cand);
                        cand &= cand - 1;
                        if (add(r, &w, a, m, k) < 0) goto fail;
                    }
                }
            }
#if ORACLE_PLANT != 1
            if (right == b) {
                /* (b, m, nn) as right operand: all k with (left, k, m) known */
                const uint64_t *ic = row(r->in, r, left, m);
                const uint64_t *ia = row(r->in, r, a, nn);
                for (int64_t wd = 0; wd < r->words; wd++) {
                    uint64_t cand = ic[wd] & ~ia[wd];
                    while (cand) {
                        int64_t k = wd * 64 + __builtin_ctzll(cand);
                        cand &= cand - 1;
                        if (add(r, &w, a, k, nn) < 0) goto fail;
                    }
                }
            }
#endif
        }
    }
    free(w.v);
    return r;
fail:
    free(w.v);
    oracle_release(r);
    return NULL;
}

int64_t oracle_count(const oracle_result *r, int32_t a) {
    if (!r || a < 0 || a >= r->n_nt) return -1;
    return r->count[a];
}

int64_t oracle_pops(const oracle_result *r) { return r ? r->pops : -1; }

/* copies R_a as (m, n) pairs sorted lexicographically; returns the number written */
int64_t oracle_copy(const oracle_result *r, int32_t a, uint32_t *pairs, int64_t cap) {
    if (!r || a < 0 || a >= r->n_nt) return -1;
    int64_t k = 0;
    for (int64_t m = 0; m < r->n; m++) {
        const uint64_t *o = row(r->out, (oracle_result *)r, a, m);
        for (int64_t wd = 0; wd < r->words; wd++) {
            uint64_t x = o[wd];
            while (x) {
                int64_t j = wd * 64 + __builtin_ctzll(x);
                x &= x - 1;
                if (k >= cap) return -1;
                pairs[2 * k] = (uint32_t)m;
                pairs[2 * k + 1] = (uint32_t)j;
                k++;
            }
        }
    }
    return k;
}

/* membership query (A, m, n) */
int oracle_has(const oracle_result *r, int32_t a, int64_t m, int64_t n) {
    if (!r || a < 0 || a >= r->n_nt || m < 0 || m >= r->n || n < 0 || n >= r->n) return -1;
    return (int)((row(r->out, (oracle_result *)r, a, m)[n >> 6] >> (n & 63)) & 1);
}
