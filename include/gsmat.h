/*
 * gsmat.h -- C ABI of libgsmat: sparse-matrix-based (SM-based) evaluation of
 * SPARQL basic graph patterns on one B300 GPU (sm_103a).
 *
 * The problem statement follows arXiv 1807.07691: an RDF dataset is a set of
 * (subject, predicate, object) triples (Sec. 3.1) stored as one sparse matrix
 * per predicate (Sec. 5.3); a basic graph pattern (BGP) is a set of triple
 * patterns whose subject and object are variables or constants and whose
 * predicate is known (Sec. 3.2, Sec. 6.3); its answer is the relation over
 * all of its variables obtained by joining the patterns' relations
 * (Sec. 6, evaluation procedure), each join being a sparse-matrix product
 * without accumulation (Sec. 6.1).
 *
 * Conventions for every call:
 *  - Return value: an int status, GSMAT_OK (0) or a GSMAT_ERR_* code.  On
 *    error no output handle is written and nothing is leaked;
 *    gsmat_last_error() gives a human-readable detail for the calling thread.
 *  - Streams: `gsmat_stream_t` is a cudaStream_t (NULL = the legacy default
 *    stream).  Work is stream-ordered; calls that return host-visible values
 *    synchronise the stream they were given.
 *  - Memory: every device buffer the library owns comes from the allocator
 *    hook (gsmat_set_allocator); the default is cudaMallocAsync/cudaFreeAsync
 *    on the call's stream.  Handles own their buffers; free them with the
 *    matching *_free call.
 *  - Ids: entity and predicate ids are int32 >= 0; entity ids and predicate
 *    ids are separate id spaces (the bijections h_so and h_p of Sec. 5.1).
 *  - Threading: a store is read-only after gsmat_load, so queries on one
 *    store may run concurrently from several host threads on different
 *    streams.  gsmat_set_allocator and gsmat_profile_* are process-global.
 *    A dictionary may be read (lookups, decoding, parsing) from several
 *    threads at once, but not while text is being added to it.
 */
#ifndef GSMAT_H_
#define GSMAT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GSMAT_API __attribute__((visibility("default")))
#else
#define GSMAT_API
#endif

typedef struct CUstream_st *gsmat_stream_t; /* == cudaStream_t */

/* Status codes. */
#define GSMAT_OK 0
#define GSMAT_ERR_INVALID_ARG 1  /* bad pointer, size, id, BGP shape or text */
#define GSMAT_ERR_UNSUPPORTED 2  /* a variable predicate (Sec. 6.3 assumes known predicates), or
                                    SPARQL beyond one basic graph pattern */
#define GSMAT_ERR_OOM 3          /* the allocator hook returned NULL (host memory, for the
                                    dictionary) */
#define GSMAT_ERR_CAPACITY 4     /* a table would exceed the library's row/offset limits */
#define GSMAT_ERR_CUDA 5         /* a CUDA runtime call failed */
#define GSMAT_ERR_DEVICE_CHECK 6 /* a kernel's own check fired (bounded wait expired) */

typedef struct gsmat_store gsmat_store; /* device-resident SM storage */
typedef struct gsmat_table gsmat_table; /* device-resident binding table */

/* ------------------------------------------------------------------------ */
/* Errors, version, allocator                                                */

/* Static description of a status code; never NULL. */
GSMAT_API const char *gsmat_strerror(int status);

/* Detail of the calling thread's last failed call ("" if none). */
GSMAT_API const char *gsmat_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
GSMAT_API int gsmat_version(void);

/* Device allocation hook.  alloc(bytes, ctx, stream) returns device memory
 * usable in stream order on `stream` (NULL on failure -> GSMAT_ERR_OOM);
 * free(ptr, ctx, stream) releases it in stream order.  Passing alloc = NULL
 * restores the default (cudaMallocAsync / cudaFreeAsync).  Process-global;
 * set it before creating stores or tables and keep it until they are freed.
 * Returns GSMAT_ERR_INVALID_ARG if exactly one of alloc/free is NULL. */
typedef void *(*gsmat_alloc_fn)(size_t bytes, void *ctx, gsmat_stream_t stream);
typedef void (*gsmat_free_fn)(void *ptr, void *ctx, gsmat_stream_t stream);
GSMAT_API int gsmat_set_allocator(gsmat_alloc_fn alloc, gsmat_free_fn free_fn, void *ctx);

/* ------------------------------------------------------------------------ */
/* SM storage (Sec. 5)                                                       */

/* Build the device store from n triples (s, p, o), row-major int32 n x 3.
 *  triples            host pointer (triples_on_device = 0; copied to the
 *                     device inside the call) or device pointer (= 1; read
 *                     only, not retained).
 *  n                  0 <= n <= 2^31 - 1.
 * The input is a multiset; duplicates are removed, since a dataset is a set
 * of triples (Sec. 3.1).  The store holds, per predicate h, the matrix M_h
 * (Sec. 5.3) twice: rows by subject (CSR) and rows by object (CSC), each
 * row's entries sorted, with the non-zero-row auxiliary arrays of Sec. 6.3
 * (row id, entry count, first position) precomputed, plus a predicate hash
 * index and the per-predicate statistics m = nnz(M_h) (Sec. 5.1, Sec. 5.3).
 * Errors: INVALID_ARG for a NULL pointer, n out of range or a negative id;
 * OOM; CUDA.  The call synchronises `stream`. */
GSMAT_API int gsmat_load(const int32_t *triples, int64_t n, int triples_on_device,
                         gsmat_stream_t stream, gsmat_store **out);

typedef struct {
    int64_t n_input;      /* triples passed to gsmat_load */
    int64_t n_unique;     /* distinct triples stored */
    int32_t n_predicates; /* distinct predicates */
    int32_t max_entity;   /* largest subject/object id (-1 if empty) */
    int32_t max_predicate;
    int32_t n_dense_rows_s; /* predicates whose CSR side uses a dense row pointer */
    int32_t n_dense_rows_o; /* same for the CSC side */
    int32_t _reserved;
    int64_t device_bytes; /* bytes held on the device by the store */
} gsmat_store_info_t;

GSMAT_API int gsmat_store_info(const gsmat_store *store, gsmat_store_info_t *info);

/* Per-predicate statistics, in ascending predicate-id order. */
typedef struct {
    int32_t pred_id; /* predicate id as given to gsmat_load */
    int32_t nnz;     /* m: number of (s, o) pairs of M_h (Sec. 5.3) */
    int32_t nr_s;    /* non-zero rows on the subject side */
    int32_t nr_o;    /* non-zero rows on the object side */
} gsmat_pred_stats;

/* Copy min(cap, n_predicates) entries into out (host); returns their count
 * through *n_out. */
GSMAT_API int gsmat_store_pred_stats(const gsmat_store *store, gsmat_pred_stats *out, int32_t cap,
                                     int32_t *n_out);

/* Copy one predicate's matrix to host buffers, for inspection and tests.
 *  side 0: rows by subject (CSR): row_ids = distinct subjects ascending,
 *          entries = objects; side 1: rows by object (CSC).
 *  row_ids   host int32[nr]       (may be NULL)
 *  row_ptr   host int64[nr + 1]   offsets into entries, row_ptr[0] = 0
 *  entries   host int32[nnz]      each row's entries ascending
 * Sizes come from gsmat_store_pred_stats.  INVALID_ARG if the predicate is
 * absent.  Synchronises `stream`. */
GSMAT_API int gsmat_store_export(const gsmat_store *store, int32_t pred_id, int side, int32_t *row_ids,
                                 int64_t *row_ptr, int32_t *entries, gsmat_stream_t stream);

/* Look up the predicate hash index on the host: slot of pred_id in the
 * ascending predicate order, or -1 if absent. */
GSMAT_API int32_t gsmat_store_pred_index(const gsmat_store *store, int32_t pred_id);

GSMAT_API void gsmat_store_free(gsmat_store *store);

/* ------------------------------------------------------------------------ */
/* BGP evaluation (Sec. 6, Alg. 1-3)                                         */

/* One triple pattern.  For each of s, p, o: *_var = 1 means the field holds
 * a variable number in 0..n_vars-1, *_var = 0 means it holds a constant id. */
typedef struct {
    int32_t s, p, o;
    uint8_t s_var, p_var, o_var, _pad;
} gsmat_pattern;

/* Query flags. */
#define GSMAT_SORTED 0u       /* columns = variables 0..V-1, rows ascending lexicographically */
#define GSMAT_PLAN_ORDER 1u   /* columns in the order the plan binds variables, rows ascending
                                 in that column order (no final sort) */
#define GSMAT_COUNT_ONLY 2u   /* compute the row count only; the table has no columns */
#define GSMAT_NO_INTERSECT 4u /* join strictly one pattern per step (Alg. 2 as printed): no
                                 fusion of an expand with a later filter into an intersection */
#define GSMAT_PLAN_COST 8u    /* plan by least estimated cost instead of Alg. 1's greedy choice
                                 (see gsmat_plan_cost); the result is the same */

/* Largest BGP that the cost-based planner searches exhaustively (larger
 * BGPs keep Alg. 1's order). */
#define GSMAT_PLAN_COST_MAX 8

/* Evaluate a BGP.
 *  pats, n_pats   host array of 1 <= n_pats <= 64 patterns.
 *  n_vars         0 <= n_vars <= 32; every variable 0..n_vars-1 must occur.
 * The plan is Alg. 1 (connected minimal upper bound) with the
 * intermediate-size estimate of Sec. 6.2 (with GSMAT_PLAN_COST, the
 * connected order of least estimated cost, gsmat_plan_cost); each step is
 * one SM-based join (Alg. 3) of the running relation with the next
 * pattern's matrix:
 * a gather-expand along the pattern's CSR or CSC rows when one end is bound,
 * a membership filter with prefix-sum compaction when both ends are bound,
 * a Cartesian product when neither is.  Result semantics: every assignment
 * of the variables that puts every pattern's triple in the store, each once
 * (no projection, no DISTINCT, no accumulation -- Sec. 6.1).
 * A predicate that is absent from the store gives an empty result.
 * Errors: INVALID_ARG (bad shape, unused or out-of-range variable, negative
 * constant), UNSUPPORTED (variable predicate), OOM, CAPACITY (more than
 * 2^32 - 1 rows in a table), CUDA, DEVICE_CHECK.  Synchronises `stream`. */
GSMAT_API int gsmat_query(const gsmat_store *store, const gsmat_pattern *pats, int n_pats, int n_vars,
                          uint32_t flags, gsmat_stream_t stream, gsmat_table **out);

/* Row sharding of one query (the rows of every step after the first are
 * independent of each other, Alg. 3): evaluate only what derives from the
 * shard-th of n_shards contiguous, near-equal parts of the first plan
 * step's relation, as gsmat_query does otherwise (same plan, flags and
 * errors; INVALID_ARG unless 0 <= shard < n_shards <= 2^20).  The shards'
 * results partition the full result: with GSMAT_PLAN_ORDER their tables
 * follow each other in shard order (concatenated, they are the full
 * table); sorted shards give the full sorted result through
 * gsmat_table_merge; COUNT_ONLY counts add up.  Shards can run on
 * different GPUs, each with a replica of the store, or one after another
 * on one GPU. */
GSMAT_API int gsmat_query_shard(const gsmat_store *store, const gsmat_pattern *pats, int n_pats, int n_vars,
                                uint32_t flags, int32_t shard, int32_t n_shards, gsmat_stream_t stream,
                                gsmat_table **out);

/* (No counterpart in the paper: the gather step of row sharding.)
 * The rows of k >= 1 tables that hold the same variables in the same column
 * order (e.g. the shards of one query), together in one new table, rows
 * ascending lexicographically in that column order: sorted tables (every
 * query result is) are merged pairwise by merge path on the device, others
 * copied back to back and reordered by all columns.  INVALID_ARG
 * for other columns or a count-only table; CAPACITY above 2^32 - 1 rows.
 * Synchronises `stream`. */
GSMAT_API int gsmat_table_merge(const gsmat_table *const *tables, int32_t k, gsmat_stream_t stream,
                                gsmat_table **out);

/* Shape of a result.  col_vars (host int32[cols], may be NULL) receives the
 * variable number held by each column. */
GSMAT_API int gsmat_table_info(const gsmat_table *table, int64_t *rows, int32_t *cols, int32_t *col_vars);

/* Device pointer to column `col` (int32[rows], owned by the table). */
GSMAT_API int gsmat_table_column(const gsmat_table *table, int32_t col, const int32_t **d_col);

/* Copy the table as row-major int32[rows][cols] into dst (host memory when
 * dst_on_device = 0, device memory otherwise).  Synchronises `stream`. */
GSMAT_API int gsmat_table_copy(const gsmat_table *table, int32_t *dst, int dst_on_device, gsmat_stream_t stream);

/* As gsmat_table_copy, but only enqueues the copy on `stream` and returns:
 * the table must stay alive and dst valid until `stream` has passed the
 * copy (e.g. until the caller synchronises it), and dst should be pinned
 * host memory for the copy to overlap other work.  Lets results of one
 * query travel to the host while the next query computes (another stream). */
GSMAT_API int gsmat_table_copy_async(const gsmat_table *table, int32_t *dst, int dst_on_device,
                                     gsmat_stream_t stream);

/* Per-query record: plan and per-step row counts. */
#define GSMAT_MAX_PATTERNS 64
typedef struct {
    int32_t n_steps;
    int32_t order[GSMAT_MAX_PATTERNS]; /* pattern index per plan step */
    int32_t kind[GSMAT_MAX_PATTERNS];  /* GSMAT_STEP_* per plan step */
    double est_rows[GSMAT_MAX_PATTERNS]; /* planner estimate after each step */
    int64_t rows[GSMAT_MAX_PATTERNS];    /* actual rows after each step */
    double est_cost;                     /* sum of est_rows */
    int64_t result_rows;
} gsmat_query_stats;

#define GSMAT_STEP_CROSS 0    /* no end bound: Cartesian product with the pattern's relation */
#define GSMAT_STEP_EXPAND_S 1 /* subject end known, object new: expand along CSR rows */
#define GSMAT_STEP_EXPAND_O 2 /* object end known, subject new: expand along CSC rows */
#define GSMAT_STEP_FILTER 3   /* both ends known: membership filter + compaction */
#define GSMAT_STEP_INTERSECT 4 /* (query stats only) an expand fused with a later filter on the
                                  new variable: the new column is the intersection of two rows */
#define GSMAT_STEP_FUSED 5     /* (query stats only) a filter executed inside an earlier INTERSECT */
#define GSMAT_STEP_PRODUCT 6   /* (query stats only) one of the plan's last steps whose lists depend
                                  only on the table before them (EXPAND from a variable bound before
                                  them or from a constant, CROSS): they run as one Cartesian product
                                  per input row, nested by variable id, so the result needs little or
                                  no final reorder; rows[] is -1 for the ones not built (exact running
                                  products when the steps start from the empty assignment).  Not used
                                  with GSMAT_NO_INTERSECT or GSMAT_PLAN_ORDER. */

GSMAT_API int gsmat_table_stats(const gsmat_table *table, gsmat_query_stats *stats);

GSMAT_API void gsmat_table_free(gsmat_table *table);

/* Projection and DISTINCT (the Select|Project form of Sec. 3.2): a new
 * table whose columns are the given variables of `table`, in the order
 * given, with every row of `table` restricted to them (distinct = 0) or
 * each such row once (distinct = 1); rows ascend lexicographically over the
 * new columns.  Runs on the device: a stable radix reorder by the new
 * columns (skipped when they are already the table's leading columns,
 * whose rows are sorted) and, for DISTINCT, a comparison of each row with
 * its predecessor and a stable compaction.
 *  vars       host int32[n], distinct variable numbers held by `table`
 *             (1 <= n <= its columns).
 * Errors: INVALID_ARG (a variable the table does not hold, a repeated one,
 * a count-only table), OOM, CUDA, DEVICE_CHECK.  Synchronises `stream`.
 * The new table is independent of `table`. */
GSMAT_API int gsmat_table_project(const gsmat_table *table, const int32_t *vars, int32_t n, int distinct,
                                  gsmat_stream_t stream, gsmat_table **out);

/* ------------------------------------------------------------------------ */
/* Batched evaluation: many BGPs in one persistent kernel                    */
/* (the same results as gsmat_query with GSMAT_SORTED, query by query)       */

typedef struct {
    const gsmat_pattern *pats; /* host array */
    int32_t n_pats;
    int32_t n_vars;
} gsmat_bgp;

typedef struct gsmat_batch gsmat_batch;

typedef struct {
    int32_t block;        /* threads per CTA: 128, 256 or 512 (0: 256) */
    int32_t ctas_per_sm;  /* persistent CTAs per SM, 1..16 (0: 4) */
    int64_t arena_bytes;  /* device arena for intermediate tables (0: 1 GiB) */
    int64_t max_rows;     /* largest table a CTA builds (0: 2^22); queries that
                             need more run on the plain path */
    int32_t use_graph;    /* 1: capture the device work as a CUDA graph */
    int32_t compact_results; /* 1: after each run, copy the results into one right-sized
                                buffer and release the arena (results then outlive the
                                arena's reuse; costs one copy of the result rows) */
    int32_t reorder_mode; /* results above 2048 rows: how their non-key columns reach the
                             reordered output when they fit a 64-bit payload (0: by size,
                             GSMAT_SORT_CARRY or GSMAT_SORT_GATHER as for gsmat_sort_rows) */
    int32_t plan_cost;    /* 0: plan every query by Alg. 1; 1: by least estimated cost, as
                             GSMAT_PLAN_COST (the results are the same) */
    int32_t expand_slots; /* tile shape of the kernel's expand loop: output slots per thread per
                             round, 1 (a search per slot) or 4 (a search per 4 consecutive slots,
                             the next parents found by stepping forward); 0: 1 */
    int32_t _pad;
} gsmat_batch_config;

typedef struct {
    int32_t n_queries;
    int32_t n_in_kernel;  /* finished inside the persistent kernel */
    int32_t n_reordered;  /* kernel result reordered by the multi-CTA sort */
    int32_t n_fallback;   /* re-run on the plain path (arena or row cap) */
    double kernel_ms;     /* device time of the last run's graph / kernel */
    double reorder_ms;    /* device time of the batched reorder of large results */
    int64_t arena_used;   /* bytes of arena the last run used */
    int32_t block;
    int32_t grid;
    int32_t n_intersect;  /* steps of the prepared programs that run as an intersect-expand (an
                             EXPAND fused with a later FILTER on its new variable) */
    int32_t _pad;
} gsmat_batch_stats_t;

/* Plan a batch of n >= 1 BGPs against a store and prepare its device run.
 * Each query is planned by Alg. 1 (Sec. 6.2; by least estimated cost when
 * cfg->plan_cost) into a step program; all
 * programs are uploaded together; the device work (queue and arena reset,
 * the persistent kernel, the copy of result descriptors) is captured as a
 * CUDA graph when cfg->use_graph (cfg may be NULL: defaults).  Validation
 * and errors as gsmat_query for every BGP.  The store must outlive the
 * batch.  Synchronises `stream`. */
GSMAT_API int gsmat_batch_prepare(const gsmat_store *store, const gsmat_bgp *bgps, int32_t n,
                                  const gsmat_batch_config *cfg, gsmat_stream_t stream, gsmat_batch **out);

/* Run (or re-run) a prepared batch.  A persistent kernel pulls query ids
 * from a device work queue; each CTA runs one query's joins at a time with
 * tables bump-allocated from the arena; queries that overflow are re-run on
 * the plain path, large results are reordered by the multi-CTA sort.  After
 * the call every result is final and valid until the next execute or free.
 * Work is ordered after prior work on `stream`, and later work on `stream`
 * is ordered after it.  Synchronises internally. */
GSMAT_API int gsmat_batch_execute(gsmat_batch *batch, gsmat_stream_t stream);

/* Shape of query i's result (columns = variables 0..V-1, rows ascending);
 * *path (may be NULL): 0 kernel, 1 plain path, 2 kernel + multi-CTA reorder. */
GSMAT_API int gsmat_batch_result(const gsmat_batch *batch, int32_t i, int64_t *rows, int32_t *cols, int32_t *path);

/* Device pointer to column `col` of query i's result (it may point into the
 * store for single-pattern results; read only). */
GSMAT_API int gsmat_batch_column(const gsmat_batch *batch, int32_t i, int32_t col, const int32_t **d_col);

/* Copy query i's result as row-major int32[rows][cols] (as gsmat_table_copy). */
GSMAT_API int gsmat_batch_copy(const gsmat_batch *batch, int32_t i, int32_t *dst, int dst_on_device,
                               gsmat_stream_t stream);

GSMAT_API int gsmat_batch_stats(const gsmat_batch *batch, gsmat_batch_stats_t *stats);

GSMAT_API void gsmat_batch_free(gsmat_batch *batch);

/* Autotuner of the persistent kernel's shape: times every (block,
 * ctas_per_sm, expand_slots) in {128, 256, 512} x {1, 2, 4, 8} x {1, 4} (at
 * most 2048 threads per SM) on the given sample batch and writes the fastest
 * into *best (the other fields come from base, which may be NULL).
 * Synchronises `stream`. */
GSMAT_API int gsmat_batch_autotune(const gsmat_store *store, const gsmat_bgp *bgps, int32_t n,
                                   const gsmat_batch_config *base, gsmat_stream_t stream, gsmat_batch_config *best);

/* Tile shapes of the plain path's join kernels on one store (the paper has
 * no counterpart: these are this library's kernel parameters). */
typedef struct {
    int32_t expand_items; /* output slots + parent rows per CTA of the expand (Alg. 3) and
                             product kernels, the size of their merge-path pieces: 512, 1024,
                             2048 (default), 4096 or 8192 */
    int32_t short_row;    /* the membership filter (Alg. 3, other join variables) searches the
                             subject's row directly when it has at most this many entries, else
                             the shorter of the subject's and the object's rows: 1..4096
                             (default 64) */
} gsmat_tiles;

/* Set / read a store's tile shapes.  Setting them while queries run on the
 * store is not allowed.  Results never depend on them.  Returns
 * GSMAT_ERR_INVALID_ARG for values outside the ranges above. */
GSMAT_API int gsmat_store_set_tiles(gsmat_store *store, const gsmat_tiles *tiles);
GSMAT_API int gsmat_store_get_tiles(const gsmat_store *store, gsmat_tiles *tiles);

/* Autotuner of the tile shapes: runs the n BGPs (a sample of the expected
 * workload) under the default shape and every shape of expand_items in
 * {512, ..., 8192} x short_row in {16, 64, 256}, each once to warm up and
 * twice timed with CUDA events on `stream`, keeps the fastest on the store
 * and writes it to *best (ties keep the default).  Synchronises `stream`;
 * no query may run on the store meanwhile. */
GSMAT_API int gsmat_store_tune(gsmat_store *store, const gsmat_bgp *bgps, int32_t n, gsmat_stream_t stream,
                               gsmat_tiles *best);

/* ------------------------------------------------------------------------ */
/* Served evaluation: continuous batching over a resident store              */

typedef struct gsmat_server gsmat_server;

typedef struct {
    int32_t max_batch;     /* queries per micro-batch (0: 1024) */
    int32_t slots;         /* micro-batches in flight at once, each on its own stream (0: 4) */
    int64_t budget_bytes;  /* admission budget: estimated device bytes of admitted, unfinished
                              requests (0: 120 GiB) */
    gsmat_batch_config batch; /* kernel shape and caps of every micro-batch (zeros: block 512,
                                 1 CTA/SM, arena up to 8 GiB sized from the estimates) */
    int32_t batch_lone;    /* 0: a request that finds the queue empty goes to an idle direct
                              lane, which runs it on the plain path (as gsmat_query, on the
                              lane's own stream and thread): under light load every request
                              starts at once on multi-CTA steps, and only requests that queue
                              up behind busy lanes form micro-batches; 1: no lanes, every
                              request is micro-batched */
    int32_t lanes;         /* direct lanes (0: 2) */
} gsmat_server_config;

typedef struct {
    int64_t submitted;
    int64_t completed;
    int64_t failed;
    int64_t batches;        /* micro-batches launched */
    int64_t fallbacks;      /* requests re-run on the plain path */
    int64_t queued;         /* now waiting for admission */
    int64_t in_flight;      /* micro-batches now on the device or being planned */
    int64_t in_flight_bytes;/* estimated bytes now admitted */
    int64_t direct;         /* requests admitted alone and run on the plain path */
} gsmat_server_stats_t;

/* Start a server over a store, which must outlive it (host threads: a
 * scheduler, a completion thread and `lanes` direct lanes).  A request that
 * finds the queue empty goes to an idle direct lane, which runs it on the
 * plain path (see batch_lone).  Otherwise the scheduler admits queued
 * requests in arrival order into a micro-batch whenever a slot is free and
 * their estimated bytes (the accumulated intermediate-size estimate of
 * Sec. 6.2 times the row width) fit in the unclaimed budget; a request
 * larger than the whole budget runs alone.  Each micro-batch is planned and
 * run as by gsmat_batch_prepare/execute on its own stream, so micro-batches
 * (and the lanes' queries) overlap on the device; a completion thread
 * finishes each as its device work ends.  The scheduler and the lanes spin
 * up to 2 ms on their next event before blocking, so at a few hundred
 * requests per second and more no request waits for a thread wake-up. */
GSMAT_API int gsmat_server_create(const gsmat_store *store, const gsmat_server_config *cfg, gsmat_server **out);

/* Queue one BGP (copied; validated as gsmat_query) and return its ticket at
 * once.  Thread-safe. */
GSMAT_API int gsmat_server_submit(gsmat_server *srv, const gsmat_pattern *pats, int n_pats, int n_vars,
                                  int64_t *ticket);

/* Wait up to timeout_us (< 0: forever) for a request; *done = 1 when its
 * result is ready.  Returns the request's error status if it failed. */
GSMAT_API int gsmat_server_wait(gsmat_server *srv, int64_t ticket, int64_t timeout_us, int32_t *done);

/* Shape of a finished request's result (as gsmat_table_info, columns =
 * variables, rows ascending) and its latency from submit to completion. */
GSMAT_API int gsmat_server_result(gsmat_server *srv, int64_t ticket, int64_t *rows, int32_t *cols,
                                  double *latency_us);

/* Copy a finished request's result (as gsmat_table_copy). */
GSMAT_API int gsmat_server_copy(gsmat_server *srv, int64_t ticket, int32_t *dst, int dst_on_device,
                                gsmat_stream_t stream);

/* Forget a finished request; its micro-batch's device memory is freed when
 * the last of its requests is released. */
GSMAT_API int gsmat_server_release(gsmat_server *srv, int64_t ticket);

GSMAT_API int gsmat_server_stats(gsmat_server *srv, gsmat_server_stats_t *stats);

/* Stop admitting, finish what is in flight, fail what is still queued, join
 * the threads and free everything (results included). */
GSMAT_API void gsmat_server_destroy(gsmat_server *srv);

/* ------------------------------------------------------------------------ */
/* String dictionary and SPARQL text (host code, no GPU needed)              */

/* Dictionary of the bijections h_p and h_so (Sec. 5.2): predicates are
 * numbered 1, 2, ... and subjects and objects share a second numbering
 * 1, 2, ..., each term by its first occurrence as triples are added, the
 * subject of a triple before its object.  Code 0 is never given out.
 *
 * Data text: statements "subject predicate object ." in the N-Triples /
 * Turtle subset: <iri>, "literal" (backslash escapes, optional @lang or
 * ^^datatype), _:blank, or a bare word (a run of bytes other than
 * whitespace and < > " { } ; , .); "@prefix p: <iri> ." declarations, after
 * which a word p:local stands for <iri local>; ';' and ',' lists; the
 * predicate word 'a' for rdf:type; '#' comments.  A term is identified by
 * its text after that prefix expansion.  A literal cannot be a subject or a
 * predicate.
 *
 * Threading: lookups, decoding and parsing may run concurrently; an add
 * may not run concurrently with anything on the same dictionary. */
typedef struct gsmat_dict gsmat_dict;

#define GSMAT_DICT_SO 0 /* subjects and objects (h_so) */
#define GSMAT_DICT_P 1  /* predicates (h_p) */

GSMAT_API int gsmat_dict_create(gsmat_dict **out);
GSMAT_API void gsmat_dict_free(gsmat_dict *dict);

/* Read the statements of text[0..len) and append their encoded triples.
 * On INVALID_ARG (bad text) or CAPACITY (more than 2^31 - 1 terms of one
 * kind) the dictionary is left as it was; after OOM (host memory) it must
 * be freed.  *n_added (may be
 * NULL) receives the number of triples read (repeated triples included:
 * gsmat_load removes them). */
GSMAT_API int gsmat_dict_add_text(gsmat_dict *dict, const char *text, int64_t len, int64_t *n_added);

/* Host threads that number the terms of an add (0, the default: one for
 * texts under 2^16 triples, else up to 16).  The codes do not depend on
 * it: terms are hashed into partitions numbered in parallel, and the codes
 * follow from the first positions of the new terms. */
GSMAT_API int gsmat_dict_set_threads(gsmat_dict *dict, int32_t n_threads);

/* All triples added so far as host int32[n][3] (s, p, o) codes, ready for
 * gsmat_load; owned by the dictionary, valid until the next add or free. */
GSMAT_API int gsmat_dict_triples(const gsmat_dict *dict, const int32_t **triples, int64_t *n);

GSMAT_API int gsmat_dict_size(const gsmat_dict *dict, int32_t *n_predicates, int32_t *n_terms);

/* Code of a term given by its identity text (prefixes expanded); 0 if the
 * dictionary does not hold it. */
GSMAT_API int gsmat_dict_lookup(const gsmat_dict *dict, int kind, const char *term, int64_t len, int32_t *code);

/* Decode n codes of one kind (ID decode): terms[i] receives a
 * NUL-terminated text owned by the dictionary (valid until it is freed),
 * lens[i] (may be NULL) its length.  INVALID_ARG for a code the dictionary
 * did not give out. */
GSMAT_API int gsmat_dict_decode(const gsmat_dict *dict, int kind, const int32_t *codes, int64_t n,
                                const char **terms, int32_t *lens);

/* A parsed SPARQL query. */
typedef struct gsmat_sparql gsmat_sparql;

/* Parse SPARQL text (the Select|Project|Join form over one BGP that
 * Sec. 3.2 shows): PREFIX declarations, SELECT [DISTINCT] followed by
 * variables (?name or $name) or '*', an optional WHERE and a brace-enclosed
 * basic graph pattern of triple patterns separated by '.', with ';' and ','
 * lists and the terms of the data text.  Variables are numbered 0, 1, ...
 * in order of first occurrence in the pattern block; '*' projects all of
 * them in that order.  Constants are coded by `dict` (a term it does not
 * hold gets code 0, which no triple has); with dict = NULL constants must
 * be decimal codes.
 * Errors: INVALID_ARG (syntax, a projected variable that no pattern uses
 * or that is repeated, more than 64 patterns or 32 variables, a literal
 * predicate); UNSUPPORTED (a variable predicate (Sec. 6.3), FILTER,
 * OPTIONAL, UNION, GRAPH, MINUS, BIND, VALUES, SERVICE, nested groups,
 * ORDER/LIMIT/OFFSET/GROUP/HAVING after the block, ASK, CONSTRUCT,
 * DESCRIBE, BASE). */
GSMAT_API int gsmat_sparql_parse(const gsmat_dict *dict, const char *text, int64_t len, gsmat_sparql **out);

/* The parsed query: its BGP (for gsmat_query), the projected variables and
 * the DISTINCT flag (for gsmat_table_project).  Pointers are owned by q. */
GSMAT_API int gsmat_sparql_info(const gsmat_sparql *q, const gsmat_pattern **pats, int32_t *n_pats, int32_t *n_vars,
                                const int32_t **proj, int32_t *n_proj, int32_t *distinct);

/* Name of variable v (without its sigil), owned by q; NULL if out of range. */
GSMAT_API const char *gsmat_sparql_var_name(const gsmat_sparql *q, int32_t v);

GSMAT_API void gsmat_sparql_free(gsmat_sparql *q);

/* ------------------------------------------------------------------------ */
/* Host planner (Alg. 1; Sec. 6.2), callable without a GPU                   */

/* Order a BGP's patterns and estimate the intermediate sizes.
 *  keys[i]    the sort statistic of pattern i: m = nnz(M_p) for a pattern
 *             without constants, the row size of its constant otherwise.
 *  stats[i]   nnz, nr_s, nr_o of pattern i's predicate (zeros if absent).
 *  order_out  int32[n_pats]: pattern index per plan step.
 *  kinds_out  int32[n_pats]: GSMAT_STEP_* per plan step (may be NULL).
 *  est_out    double[n_pats]: running estimate after each step (may be NULL).
 * Stable sort by key, then repeatedly the first remaining pattern sharing a
 * variable with those taken (the smallest remaining one if none does).
 * The estimate multiplies, per step: CROSS -> key; EXPAND from a constant ->
 * key; EXPAND from a bound variable -> nnz / nr on that side; FILTER ->
 * min(1, nnz / (nr_s * nr_o)); starting from 1. */
GSMAT_API int gsmat_plan(const gsmat_pattern *pats, int n_pats, int n_vars, const int64_t *keys,
                         const gsmat_pred_stats *stats, int32_t *order_out, int32_t *kinds_out,
                         double *est_out);

/* Cost-based variant (Thm. 2 makes the accumulated estimate the quantity a
 * plan should keep small; Alg. 1 only approximates its minimum greedily).
 * Same arguments and outputs as gsmat_plan.  Among the connected orders --
 * orders in which every step takes a pattern sharing a variable with the
 * patterns before it, unless no remaining pattern does -- returns one whose
 * cost (sum of the running estimates, computed as gsmat_plan computes them)
 * is least; among equal costs, the one that comes first when orders are
 * compared as sequences of positions in the stable key order, so Alg. 1's
 * order (itself connected) is kept on a tie.  Exhaustive with pruning for
 * n_pats <= GSMAT_PLAN_COST_MAX (at most 8! orders), Alg. 1 above that.
 * Never costs more than gsmat_plan's order.  Errors as gsmat_plan. */
GSMAT_API int gsmat_plan_cost(const gsmat_pattern *pats, int n_pats, int n_vars, const int64_t *keys,
                              const gsmat_pred_stats *stats, int32_t *order_out, int32_t *kinds_out,
                              double *est_out);

/* ------------------------------------------------------------------------ */
/* Device primitives used by the store builder and the join (exported so     */
/* that they can be tested and reused on their own)                          */

/* Stable LSD radix sort of n uint64 keys on bits [begin_bit, end_bit),
 * 8 bits per pass, with an optional uint32 payload (d_vals may be NULL).
 * d_keys / d_vals are device arrays, sorted in place.  0 <= n < 2^32.
 * Scratch comes from the allocator hook.  Does not synchronise, so a
 * bounded wait that expires inside (a predecessor tile that never publishes
 * its counts) is not reported: the output is then unspecified. */
GSMAT_API int gsmat_radix_sort_u64(uint64_t *d_keys, uint32_t *d_vals, int64_t n, int begin_bit, int end_bit,
                                   gsmat_stream_t stream);

/* Canonical output of a binding table (the result row of Sec. 6.3 over the
 * variables in id order): stable lexicographic reorder of n rows by their
 * first m of V columns.  d_cols[v] / d_out[v] (v < V) are device int32
 * columns of n rows; every value must lie in [0, 2^bits).  Keys pack
 * floor(64 / bits) columns each; wider orders sort chunk by chunk, least
 * significant first, each chunk being 8-bit onesweep passes whose first pass
 * packs the keys from the columns and whose last pass writes d_out.
 * 1 <= m <= V <= 32, 1 <= bits <= 31, 0 <= n < 2^32; d_out must not alias
 * d_cols.  Scratch comes from the allocator hook.  Does not synchronise, so a
 * bounded wait that expires inside is not reported (output unspecified). */
GSMAT_API int gsmat_sort_rows(const int32_t *const *d_cols, int V, int m, int bits, int64_t n,
                              int32_t *const *d_out, uint32_t flags, gsmat_stream_t stream);
/* flags of gsmat_sort_rows: how the other V - m columns reach d_out when
 * they fit one 64-bit payload, the key one word, and n > 2048 (0: chosen by
 * size) */
#define GSMAT_SORT_CARRY 1u  /* carried through the passes beside the key */
#define GSMAT_SORT_GATHER 2u /* gathered through the sorted row index */

/* Exclusive prefix sum of n int32 counts (each >= 0) into d_out[0..n]
 * (int64; d_out[n] = total), single pass with decoupled look-back over
 * tiles.  Scratch (tile descriptors) comes from the allocator hook.
 * Does not synchronise, so a bounded wait that expires inside is not
 * reported (output unspecified). */
GSMAT_API int gsmat_exclusive_scan_i32(const int32_t *d_in, int64_t *d_out, int64_t n, gsmat_stream_t stream);

/* The same exclusive prefix sum, for callers that cannot allocate device
 * memory: code that runs under a fixed device-memory budget already handed
 * out to another allocator, or on a latency-critical path that must not
 * enter the driver's allocator (which can block and synchronise the device).
 * The paper has no counterpart; this is a library convenience.
 *  - Allocates nothing: no cudaMalloc/cudaFree, no allocator hook.  The tile
 *    descriptors live in a file-scope static device array of 256 KB (plus
 *    32 bytes), which every GPU that loads the library holds until the
 *    process exits.
 *  - n <= gsmat_exclusive_scan_i32_noalloc_max() (2^26 = 67,108,864);
 *    larger n returns GSMAT_ERR_CAPACITY without touching the device.
 *  - The first call on a device looks the array's device address up once
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept for the rest of the
 *    process: it does not survive cudaDeviceReset (which reloads the
 *    library's device code), so do not call this after a device reset.
 *  - Every call shares the array and clears the part it uses (stream-ordered
 *    memsets) before its kernel; calls whose work overlaps on the GPU (other
 *    streams, other host threads) race on it and must be serialised by the
 *    caller.
 *  - d_in, d_out: device arrays as for gsmat_exclusive_scan_i32.  n = 0
 *    writes d_out[0] = 0.
 *  - Does not synchronise, so a bounded wait that expires inside is not
 *    reported (output unspecified); the error word it sets in the array is
 *    cleared by the next call. */
GSMAT_API int gsmat_exclusive_scan_i32_noalloc(const int32_t *d_in, int64_t *d_out, int64_t n,
                                               gsmat_stream_t stream);
GSMAT_API int64_t gsmat_exclusive_scan_i32_noalloc_max(void);

/* Self-test of the kernels' bounded waits (failure detection without a GPU
 * fault).  Runs the library's single-pass scan kernel -- the look-back code
 * of a query's count, scan and compaction steps -- over four tiles of zeros
 * with its tile counter starting at 1: tile 0 never runs, so the look-back
 * of every other tile waits on a descriptor that nothing writes.  After
 * poll_limit polls (1 <= poll_limit <= 2^22; each poll sleeps about 64 ns)
 * each wait gives up, records the error word and lets its CTA finish; the
 * call then synchronises `stream` and reads the word.
 * Returns GSMAT_ERR_DEVICE_CHECK when the waits expired (the designed
 * outcome; the device and the stream stay usable), GSMAT_OK if they did
 * not (a defect), GSMAT_ERR_INVALID_ARG for a poll limit out of range.
 * The paper has no counterpart: this checks the library's own failure
 * handling. */
GSMAT_API int gsmat_selftest_wait_expiry(int32_t poll_limit, gsmat_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Kernel timing (CUDA events on the launching stream)                       */

typedef struct {
    char name[32];         /* kernel family */
    int64_t launches;      /* timed calls of the family (each may launch several kernels) */
    double total_ms;       /* sum of event-timed durations */
    double algo_bytes;     /* sum of algorithmic bytes moved (see docs per kernel) */
    double items;          /* sum of items processed (rows or keys) */
} gsmat_kernel_profile;

/* Enable (1) or disable (0) per-launch event timing in all later calls. */
GSMAT_API int gsmat_profile_enable(int on);

/* Copy up to cap kernel families into out; *n_out gets their count.
 * reset = 1 clears the counters after reading. */
GSMAT_API int gsmat_profile_read(gsmat_kernel_profile *out, int32_t cap, int32_t *n_out, int reset);

/* Number of CUDA kernels the library has launched since it was loaded (all
 * threads; monotonic).  Never fails. */
GSMAT_API int64_t gsmat_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* GSMAT_H_ */
