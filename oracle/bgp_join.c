/*
 * Oracle for basic-graph-pattern evaluation -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may call this code.  It shares nothing with the CUDA path.
 *
 * What it computes (Sec. 6, "procedure of SM-based BGP query evaluation",
 * and Sec. 6.1, join as sparse-matrix multiplication without accumulation):
 * given a triple *set* D (Sec. 3.1) and a BGP of patterns (s, p, o) whose s
 * and o are variables or constants and whose p is a constant (Sec. 6.3), the
 * result is every assignment mu of the BGP's variables to entity ids such
 * that (mu(s), p, mu(o)) is in D for every pattern, constants mapping to
 * themselves.  All variables are kept (no projection, no accumulation), so
 * the result is a relation over variables 0..V-1; it is returned as rows
 * sorted lexicographically in variable order.
 *
 * How: the plain definition, evaluated as a left-deep nested-loop join in
 * the patterns' INPUT order (deliberately not a planned order).  The triple
 * set is sorted twice, by (p, s, o) and by (p, o, s), and probed by binary
 * search: a pattern with both ends known is a membership probe, with one end
 * known a range scan of the matching (p, s, *) or (p, *, o) block, and with
 * neither known a scan of the whole (p, *, *) block (which makes a Cartesian
 * product with the rows so far when the pattern shares no variable).  A
 * repeated variable (?x p ?x) only matches triples with s == o.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_INVALID 1
#define ORACLE_ERR_UNSUPPORTED 2
#define ORACLE_ERR_ROW_LIMIT 3
#define ORACLE_ERR_OOM 4

typedef struct {
    int32_t s, p, o;
} triple_t;

static int cmp_pso(const void *a, const void *b) {
    const triple_t *x = (const triple_t *)a, *y = (const triple_t *)b;
    if (x->p != y->p) return x->p < y->p ? -1 : 1;
    if (x->s != y->s) return x->s < y->s ? -1 : 1;
    if (x->o != y->o) return x->o < y->o ? -1 : 1;
    return 0;
}

static int cmp_pos(const void *a, const void *b) {
    const triple_t *x = (const triple_t *)a, *y = (const triple_t *)b;
    if (x->p != y->p) return x->p < y->p ? -1 : 1;
    if (x->o != y->o) return x->o < y->o ? -1 : 1;
    if (x->s != y->s) return x->s < y->s ? -1 : 1;
    return 0;
}

/* The triple set, indexed two ways. */
typedef struct {
    triple_t *pso; /* sorted by (p, s, o), duplicates removed */
    triple_t *pos; /* the same set sorted by (p, o, s) */
    int64_t n;
} oracle_index_t;

/* First position in t[0..n) whose key is >= (p, a) where a is the second
 * sort field (s for pso, o for pos); use_a = 0 searches on p alone. */
static int64_t lower(const triple_t *t, int64_t n, int32_t p, int32_t a, int use_a, int by_o) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int32_t mp = t[mid].p;
        int32_t ma = by_o ? t[mid].o : t[mid].s;
        int less = (mp < p) || (use_a && mp == p && ma < a);
        if (less) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* First position whose key is > (p, a) (or > p when use_a = 0). */
static int64_t upper(const triple_t *t, int64_t n, int32_t p, int32_t a, int use_a, int by_o) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int32_t mp = t[mid].p;
        int32_t ma = by_o ? t[mid].o : t[mid].s;
        int le = (mp < p) || (mp == p && (!use_a || ma <= a));
        if (le) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int contains(const oracle_index_t *ix, int32_t s, int32_t p, int32_t o) {
    triple_t key = {s, p, o};
    return bsearch(&key, ix->pso, (size_t)ix->n, sizeof(triple_t), cmp_pso) != NULL;
}

int oracle_index_build(const int32_t *triples, int64_t n, oracle_index_t **out) {
    oracle_index_t *ix = (oracle_index_t *)calloc(1, sizeof(*ix));
    if (!ix) return ORACLE_ERR_OOM;
    ix->pso = (triple_t *)malloc(sizeof(triple_t) * (size_t)(n > 0 ? n : 1));
    ix->pos = (triple_t *)malloc(sizeof(triple_t) * (size_t)(n > 0 ? n : 1));
    if (!ix->pso || !ix->pos) {
        free(ix->pso); free(ix->pos); free(ix);
        return ORACLE_ERR_OOM;
    }
    for (int64_t i = 0; i < n; i++) {
        ix->pso[i].s = triples[3 * i + 0];
        ix->pso[i].p = triples[3 * i + 1];
        ix->pso[i].o = triples[3 * i + 2];
    }
    qsort(ix->pso, (size_t)n, sizeof(triple_t), cmp_pso);
    /* D is a set (Sec. 3.1): drop repeated triples. */
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
        if (m == 0 || cmp_pso(&ix->pso[m - 1], &ix->pso[i]) != 0) ix->pso[m++] = ix->pso[i];
    }
    ix->n = m;
    memcpy(ix->pos, ix->pso, sizeof(triple_t) * (size_t)m);
    qsort(ix->pos, (size_t)m, sizeof(triple_t), cmp_pos);
    *out = ix;
    return ORACLE_OK;
}

void oracle_index_free(oracle_index_t *ix) {
    if (!ix) return;
    free(ix->pso);
    free(ix->pos);
    free(ix);
}

int64_t oracle_index_size(const oracle_index_t *ix) { return ix->n; }

/* A growable table of rows, each n_vars int32 wide (unbound slots hold -1). */
typedef struct {
    int32_t *data;
    int64_t rows, cap;
    int width;
} table_t;

static int table_push(table_t *t, const int32_t *row) {
    if (t->rows == t->cap) {
        int64_t ncap = t->cap ? t->cap * 2 : 1024;
        size_t bytes = (size_t)ncap * (size_t)(t->width > 0 ? t->width : 1) * sizeof(int32_t);
        int32_t *nd = (int32_t *)realloc(t->data, bytes);
        if (!nd) return ORACLE_ERR_OOM;
        t->data = nd;
        t->cap = ncap;
    }
    if (t->width > 0) memcpy(t->data + t->rows * t->width, row, sizeof(int32_t) * (size_t)t->width);
    t->rows++;
    return ORACLE_OK;
}

static int g_sort_width; /* the oracle is single-threaded */
static int cmp_rows(const void *a, const void *b) {
    const int32_t *x = (const int32_t *)a, *y = (const int32_t *)b;
    for (int i = 0; i < g_sort_width; i++) {
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    }
    return 0;
}

/*
 * Evaluate one BGP.  pats is n_pats x 6 int64: s, p, o, s_is_var, p_is_var,
 * o_is_var; a variable end holds its variable number in 0..n_vars-1.
 * On success *rows_out (malloc'ed, caller frees with oracle_free) holds
 * *n_rows_out rows of n_vars int32 in lexicographic order; step_rows (may be
 * NULL) receives the row count after each pattern, in input order.
 * Returns ORACLE_ERR_ROW_LIMIT as soon as a table would exceed row_limit.
 */
int oracle_bgp(const oracle_index_t *ix, const int64_t *pats, int n_pats, int n_vars,
               int64_t row_limit, int32_t **rows_out, int64_t *n_rows_out, int64_t *step_rows) {
    *rows_out = NULL;
    *n_rows_out = 0;
    if (n_pats <= 0 || n_vars < 0) return ORACLE_ERR_INVALID;
    /* every variable 0..n_vars-1 must occur; ids must be valid */
    char *used = (char *)calloc((size_t)(n_vars > 0 ? n_vars : 1), 1);
    if (!used) return ORACLE_ERR_OOM;
    for (int k = 0; k < n_pats; k++) {
        const int64_t *q = pats + 6 * k;
        if (q[4]) { free(used); return ORACLE_ERR_UNSUPPORTED; }
        for (int e = 0; e < 3; e += 2) {
            if (q[3 + e]) {
                if (q[e] < 0 || q[e] >= n_vars) { free(used); return ORACLE_ERR_INVALID; }
                used[q[e]] = 1;
            } else if (q[e] < 0 || q[e] > INT32_MAX) {
                free(used); return ORACLE_ERR_INVALID;
            }
        }
        if (q[1] < 0 || q[1] > INT32_MAX) { free(used); return ORACLE_ERR_INVALID; }
    }
    for (int v = 0; v < n_vars; v++) {
        if (!used[v]) { free(used); return ORACLE_ERR_INVALID; }
    }
    free(used);

    char *bound = (char *)calloc((size_t)(n_vars > 0 ? n_vars : 1), 1);
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_vars > 0 ? n_vars : 1));
    table_t cur = {0}, nxt = {0};
    cur.width = nxt.width = n_vars;
    int rc = ORACLE_OK;
    if (!bound || !row) { rc = ORACLE_ERR_OOM; goto done; }
    /* Start from the relation with one empty assignment. */
    for (int v = 0; v < n_vars; v++) row[v] = -1;
    if ((rc = table_push(&cur, row))) goto done;

    for (int k = 0; k < n_pats; k++) {
        const int64_t *q = pats + 6 * k;
        const int32_t p = (int32_t)q[1];
        const int s_var = (int)q[3], o_var = (int)q[5];
        const int s_id = (int)q[0], o_id = (int)q[2];
        const int same_var = s_var && o_var && s_id == o_id;
        nxt.rows = 0;
        for (int64_t r = 0; r < cur.rows; r++) {
            const int32_t *in = cur.data + r * n_vars;
            int s_known = !s_var || bound[s_id];
            int o_known = !o_var || bound[o_id];
            int32_t s_val = s_var ? (s_known ? in[s_id] : -1) : (int32_t)q[0];
            int32_t o_val = o_var ? (o_known ? in[o_id] : -1) : (int32_t)q[2];
            if (n_vars > 0) memcpy(row, in, sizeof(int32_t) * (size_t)n_vars);
            if (s_known && o_known) {
                if (contains(ix, s_val, p, o_val)) {
                    if ((rc = table_push(&nxt, row))) goto done;
                }
            } else if (s_known) {
                int64_t a = lower(ix->pso, ix->n, p, s_val, 1, 0);
                int64_t b = upper(ix->pso, ix->n, p, s_val, 1, 0);
                for (int64_t i = a; i < b; i++) {
                    row[o_id] = ix->pso[i].o;
                    if ((rc = table_push(&nxt, row))) goto done;
                }
            } else if (o_known) {
                int64_t a = lower(ix->pos, ix->n, p, o_val, 1, 1);
                int64_t b = upper(ix->pos, ix->n, p, o_val, 1, 1);
                for (int64_t i = a; i < b; i++) {
                    row[s_id] = ix->pos[i].s;
                    if ((rc = table_push(&nxt, row))) goto done;
                }
            } else {
                int64_t a = lower(ix->pso, ix->n, p, 0, 0, 0);
                int64_t b = upper(ix->pso, ix->n, p, 0, 0, 0);
                for (int64_t i = a; i < b; i++) {
                    if (same_var && ix->pso[i].s != ix->pso[i].o) continue;
                    row[s_id] = ix->pso[i].s;
                    row[o_id] = ix->pso[i].o;
                    if ((rc = table_push(&nxt, row))) goto done;
                }
            }
            if (nxt.rows > row_limit) { rc = ORACLE_ERR_ROW_LIMIT; goto done; }
        }
        if (s_var) bound[s_id] = 1;
        if (o_var) bound[o_id] = 1;
        if (step_rows) step_rows[k] = nxt.rows;
        table_t tmp = cur; cur = nxt; nxt = tmp;
    }
    if (n_vars > 0 && cur.rows > 1) {
        g_sort_width = n_vars;
        qsort(cur.data, (size_t)cur.rows, sizeof(int32_t) * (size_t)n_vars, cmp_rows);
    }
    *n_rows_out = cur.rows;
    if (n_vars > 0 && cur.rows > 0) {
        *rows_out = cur.data;
        cur.data = NULL;
    }
done:
    free(cur.data);
    free(nxt.data);
    free(bound);
    free(row);
    return rc;
}

void oracle_free(void *p) { free(p); }
