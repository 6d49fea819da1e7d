// The C ABI of libgsmat (include/gsmat.h): argument checks and dispatch.
#include <string.h>

#include <new>

#include "dict.h"
#include "join.cuh"
#include "plan.h"
#include "query.cuh"
#include "store.cuh"

namespace gs {
int batch_prepare(const gsmat_store *S, const gsmat_bgp *bgps, int32_t n, const gsmat_batch_config *cfg,
                  cudaStream_t st, gsmat_batch **out);
int batch_execute(gsmat_batch *B, cudaStream_t st);
int batch_result(const gsmat_batch *B, int32_t i, int64_t *rows, int32_t *cols, int32_t *path);
int batch_column(const gsmat_batch *B, int32_t i, int32_t c, const int32_t **d_col);
int batch_copy(const gsmat_batch *B, int32_t i, int32_t *dst, int dst_on_device, cudaStream_t st);
int batch_stats(const gsmat_batch *B, gsmat_batch_stats_t *s);
int batch_autotune(const gsmat_store *S, const gsmat_bgp *bgps, int32_t n, const gsmat_batch_config *base,
                   cudaStream_t st, gsmat_batch_config *best);
void batch_free(gsmat_batch *B);
int server_create(const gsmat_store *S, const gsmat_server_config *cfg, gsmat_server **out);
int server_submit(gsmat_server *srv, const gsmat_pattern *pats, int n_pats, int n_vars, int64_t *ticket);
int server_wait(gsmat_server *srv, int64_t ticket, int64_t timeout_us, int32_t *done);
int server_result(gsmat_server *srv, int64_t ticket, int64_t *rows, int32_t *cols, double *latency_us);
int server_copy(gsmat_server *srv, int64_t ticket, int32_t *dst, int dst_on_device, cudaStream_t st);
int server_release(gsmat_server *srv, int64_t ticket);
int server_stats(gsmat_server *srv, gsmat_server_stats_t *s);
void server_destroy(gsmat_server *srv);
const char *last_error();
int set_allocator(gsmat_alloc_fn a, gsmat_free_fn f, void *ctx);
int profile_enable(int on);
int profile_read(gsmat_kernel_profile *out, int32_t cap, int32_t *n_out, int reset);
int64_t launch_count();
}  // namespace gs

using gs::set_error;

extern "C" {

GSMAT_API const char *gsmat_strerror(int status) {
    switch (status) {
        case GSMAT_OK: return "ok";
        case GSMAT_ERR_INVALID_ARG: return "invalid argument";
        case GSMAT_ERR_UNSUPPORTED: return "unsupported (variable predicate)";
        case GSMAT_ERR_OOM: return "out of device memory";
        case GSMAT_ERR_CAPACITY: return "capacity exceeded";
        case GSMAT_ERR_CUDA: return "CUDA error";
        case GSMAT_ERR_DEVICE_CHECK: return "device-side check failed";
        default: return "unknown status";
    }
}

GSMAT_API const char *gsmat_last_error(void) { return gs::last_error(); }

GSMAT_API int gsmat_version(void) { return 100; }

GSMAT_API int gsmat_set_allocator(gsmat_alloc_fn alloc, gsmat_free_fn free_fn, void *ctx) {
    gs::clear_error();
    return gs::set_allocator(alloc, free_fn, ctx);
}

GSMAT_API int gsmat_load(const int32_t *triples, int64_t n, int triples_on_device, gsmat_stream_t stream,
                         gsmat_store **out) {
    gs::clear_error();
    return gs::store_build(triples, n, triples_on_device, (cudaStream_t)stream, out);
}

GSMAT_API int gsmat_store_info(const gsmat_store *S, gsmat_store_info_t *info) {
    gs::clear_error();
    if (!S || !info) return set_error(GSMAT_ERR_INVALID_ARG, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->n_input = S->n_input;
    info->n_unique = S->n_unique;
    info->n_predicates = S->n_pred;
    info->max_entity = S->max_entity;
    info->max_predicate = S->max_pred;
    info->n_dense_rows_s = S->n_dense[0];
    info->n_dense_rows_o = S->n_dense[1];
    info->device_bytes = S->device_bytes();
    return GSMAT_OK;
}

GSMAT_API int gsmat_store_pred_stats(const gsmat_store *S, gsmat_pred_stats *out, int32_t cap, int32_t *n_out) {
    gs::clear_error();
    if (!S || (!out && cap > 0)) return set_error(GSMAT_ERR_INVALID_ARG, "NULL argument");
    const int32_t n = S->n_pred < cap ? S->n_pred : cap;
    for (int32_t i = 0; i < n; ++i) {
        out[i].pred_id = S->pred_ids[i];
        out[i].nnz = S->side[0][i].nnz;
        out[i].nr_s = S->side[0][i].nrows;
        out[i].nr_o = S->side[1][i].nrows;
    }
    if (n_out) *n_out = n;
    return GSMAT_OK;
}

GSMAT_API int32_t gsmat_store_pred_index(const gsmat_store *S, int32_t pred_id) {
    if (!S) return -1;
    return S->slot_of(pred_id);
}

GSMAT_API int gsmat_store_export(const gsmat_store *S, int32_t pred_id, int side, int32_t *row_ids, int64_t *row_ptr,
                                 int32_t *entries, gsmat_stream_t stream) {
    gs::clear_error();
    if (!S || (side != 0 && side != 1)) return set_error(GSMAT_ERR_INVALID_ARG, "bad store or side");
    const int32_t slot = S->slot_of(pred_id);
    if (slot < 0) return set_error(GSMAT_ERR_INVALID_ARG, "predicate %d not in the store", pred_id);
    cudaStream_t st = (cudaStream_t)stream;
    const gs::PredSide &ps = S->side[side][slot];
    std::vector<int32_t> off((size_t)ps.nrows + 1);
    if (row_ids && ps.nrows > 0) {
        GS_CUDA(cudaMemcpyAsync(row_ids, S->rowid[side].as<int32_t>() + ps.row_base, sizeof(int32_t) * ps.nrows,
                                cudaMemcpyDeviceToHost, st));
    }
    GS_CUDA(cudaMemcpyAsync(off.data(), S->rowoff[side].as<int32_t>() + ps.row_base, sizeof(int32_t) * (ps.nrows + 1),
                            cudaMemcpyDeviceToHost, st));
    if (entries && ps.nnz > 0) {
        GS_CUDA(cudaMemcpyAsync(entries, S->val[side].as<int32_t>() + ps.ent_base, sizeof(int32_t) * ps.nnz,
                                cudaMemcpyDeviceToHost, st));
    }
    GS_CUDA(cudaStreamSynchronize(st));
    if (row_ptr) {
        for (int32_t r = 0; r <= ps.nrows; ++r) row_ptr[r] = (int64_t)off[r] - ps.ent_base;
    }
    return GSMAT_OK;
}

GSMAT_API void gsmat_store_free(gsmat_store *S) { delete S; }

GSMAT_API int gsmat_query(const gsmat_store *S, const gsmat_pattern *pats, int n_pats, int n_vars, uint32_t flags,
                          gsmat_stream_t stream, gsmat_table **out) {
    gs::clear_error();
    return gs::query_run(S, pats, n_pats, n_vars, flags, (cudaStream_t)stream, out);
}

GSMAT_API int gsmat_table_info(const gsmat_table *T, int64_t *rows, int32_t *cols, int32_t *col_vars) {
    gs::clear_error();
    if (!T) return set_error(GSMAT_ERR_INVALID_ARG, "table is NULL");
    if (rows) *rows = T->rows;
    if (cols) *cols = T->ncols;
    if (col_vars) {
        for (int c = 0; c < T->ncols; ++c) col_vars[c] = T->vars[c];
    }
    return GSMAT_OK;
}

GSMAT_API int gsmat_table_column(const gsmat_table *T, int32_t col, const int32_t **d_col) {
    gs::clear_error();
    if (!T || !d_col || col < 0 || col >= T->ncols) return set_error(GSMAT_ERR_INVALID_ARG, "bad table or column");
    *d_col = T->col[col];
    return GSMAT_OK;
}

GSMAT_API int gsmat_table_copy(const gsmat_table *T, int32_t *dst, int dst_on_device, gsmat_stream_t stream) {
    gs::clear_error();
    return gs::table_copy(T, dst, dst_on_device, (cudaStream_t)stream);
}

GSMAT_API int gsmat_table_copy_async(const gsmat_table *T, int32_t *dst, int dst_on_device,
                                     gsmat_stream_t stream) {
    gs::clear_error();
    return gs::table_copy(T, dst, dst_on_device, (cudaStream_t)stream, false);
}

GSMAT_API int gsmat_table_stats(const gsmat_table *T, gsmat_query_stats *stats) {
    gs::clear_error();
    if (!T || !stats) return set_error(GSMAT_ERR_INVALID_ARG, "NULL argument");
    *stats = T->stats;
    return GSMAT_OK;
}

GSMAT_API void gsmat_table_free(gsmat_table *T) { delete T; }

GSMAT_API int gsmat_batch_prepare(const gsmat_store *store, const gsmat_bgp *bgps, int32_t n,
                                  const gsmat_batch_config *cfg, gsmat_stream_t stream, gsmat_batch **out) {
    gs::clear_error();
    return gs::batch_prepare(store, bgps, n, cfg, (cudaStream_t)stream, out);
}

GSMAT_API int gsmat_batch_execute(gsmat_batch *batch, gsmat_stream_t stream) {
    gs::clear_error();
    return gs::batch_execute(batch, (cudaStream_t)stream);
}

GSMAT_API int gsmat_batch_result(const gsmat_batch *batch, int32_t i, int64_t *rows, int32_t *cols, int32_t *path) {
    gs::clear_error();
    return gs::batch_result(batch, i, rows, cols, path);
}

GSMAT_API int gsmat_batch_column(const gsmat_batch *batch, int32_t i, int32_t col, const int32_t **d_col) {
    gs::clear_error();
    return gs::batch_column(batch, i, col, d_col);
}

GSMAT_API int gsmat_batch_copy(const gsmat_batch *batch, int32_t i, int32_t *dst, int dst_on_device,
                               gsmat_stream_t stream) {
    gs::clear_error();
    return gs::batch_copy(batch, i, dst, dst_on_device, (cudaStream_t)stream);
}

GSMAT_API int gsmat_batch_stats(const gsmat_batch *batch, gsmat_batch_stats_t *stats) {
    gs::clear_error();
    return gs::batch_stats(batch, stats);
}

GSMAT_API void gsmat_batch_free(gsmat_batch *batch) { gs::batch_free(batch); }

GSMAT_API int gsmat_batch_autotune(const gsmat_store *store, const gsmat_bgp *bgps, int32_t n,
                                   const gsmat_batch_config *base, gsmat_stream_t stream, gsmat_batch_config *best) {
    gs::clear_error();
    return gs::batch_autotune(store, bgps, n, base, (cudaStream_t)stream, best);
}

GSMAT_API int gsmat_server_create(const gsmat_store *store, const gsmat_server_config *cfg, gsmat_server **out) {
    gs::clear_error();
    return gs::server_create(store, cfg, out);
}

GSMAT_API int gsmat_server_submit(gsmat_server *srv, const gsmat_pattern *pats, int n_pats, int n_vars,
                                  int64_t *ticket) {
    gs::clear_error();
    return gs::server_submit(srv, pats, n_pats, n_vars, ticket);
}

GSMAT_API int gsmat_server_wait(gsmat_server *srv, int64_t ticket, int64_t timeout_us, int32_t *done) {
    gs::clear_error();
    return gs::server_wait(srv, ticket, timeout_us, done);
}

GSMAT_API int gsmat_server_result(gsmat_server *srv, int64_t ticket, int64_t *rows, int32_t *cols,
                                  double *latency_us) {
    gs::clear_error();
    return gs::server_result(srv, ticket, rows, cols, latency_us);
}

GSMAT_API int gsmat_server_copy(gsmat_server *srv, int64_t ticket, int32_t *dst, int dst_on_device,
                                gsmat_stream_t stream) {
    gs::clear_error();
    if (!srv) return set_error(GSMAT_ERR_INVALID_ARG, "server is NULL");
    return gs::server_copy(srv, ticket, dst, dst_on_device, (cudaStream_t)stream);
}

GSMAT_API int gsmat_server_release(gsmat_server *srv, int64_t ticket) {
    gs::clear_error();
    if (!srv) return set_error(GSMAT_ERR_INVALID_ARG, "server is NULL");
    return gs::server_release(srv, ticket);
}

GSMAT_API int gsmat_server_stats(gsmat_server *srv, gsmat_server_stats_t *stats) {
    gs::clear_error();
    return gs::server_stats(srv, stats);
}

GSMAT_API void gsmat_server_destroy(gsmat_server *srv) { gs::server_destroy(srv); }

GSMAT_API int gsmat_plan(const gsmat_pattern *pats, int n_pats, int n_vars, const int64_t *keys,
                         const gsmat_pred_stats *stats, int32_t *order_out, int32_t *kinds_out, double *est_out) {
    gs::clear_error();
    GS_TRY(gs::validate_bgp(pats, n_pats, n_vars));
    if (!keys || !stats || !order_out) return set_error(GSMAT_ERR_INVALID_ARG, "NULL argument");
    return gs::plan_bgp(pats, n_pats, keys, stats, order_out, kinds_out, est_out);
}

GSMAT_API int gsmat_query_shard(const gsmat_store *store, const gsmat_pattern *pats, int n_pats, int n_vars,
                                uint32_t flags, int32_t shard, int32_t n_shards, gsmat_stream_t stream,
                                gsmat_table **out) {
    gs::clear_error();
    return gs::query_run(store, pats, n_pats, n_vars, flags, (cudaStream_t)stream, out, shard, n_shards);
}

GSMAT_API int gsmat_table_merge(const gsmat_table *const *tables, int32_t k, gsmat_stream_t stream,
                                gsmat_table **out) {
    gs::clear_error();
    return gs::table_merge(tables, k, (cudaStream_t)stream, out);
}

GSMAT_API int gsmat_table_project(const gsmat_table *table, const int32_t *vars, int32_t n, int distinct,
                                  gsmat_stream_t stream, gsmat_table **out) {
    gs::clear_error();
    return gs::table_project(table, vars, n, distinct, (cudaStream_t)stream, out);
}

GSMAT_API int gsmat_dict_create(gsmat_dict **out) {
    gs::clear_error();
    return gs::dict_create(out);
}

GSMAT_API void gsmat_dict_free(gsmat_dict *dict) { gs::dict_free(dict); }

GSMAT_API int gsmat_dict_set_threads(gsmat_dict *dict, int32_t n_threads) {
    gs::clear_error();
    return gs::dict_set_threads(dict, n_threads);
}

GSMAT_API int gsmat_dict_add_text(gsmat_dict *dict, const char *text, int64_t len, int64_t *n_added) {
    gs::clear_error();
    try {
        return gs::dict_add_text(dict, text, len, n_added);
    } catch (const std::bad_alloc &) {
        return set_error(GSMAT_ERR_OOM, "host memory ran out while adding text (free the dictionary)");
    }
}

GSMAT_API int gsmat_dict_triples(const gsmat_dict *dict, const int32_t **triples, int64_t *n) {
    gs::clear_error();
    return gs::dict_triples(dict, triples, n);
}

GSMAT_API int gsmat_dict_size(const gsmat_dict *dict, int32_t *n_predicates, int32_t *n_terms) {
    gs::clear_error();
    return gs::dict_size(dict, n_predicates, n_terms);
}

GSMAT_API int gsmat_dict_lookup(const gsmat_dict *dict, int kind, const char *term, int64_t len, int32_t *code) {
    gs::clear_error();
    return gs::dict_lookup(dict, kind, term, len, code);
}

GSMAT_API int gsmat_dict_decode(const gsmat_dict *dict, int kind, const int32_t *codes, int64_t n,
                                const char **terms, int32_t *lens) {
    gs::clear_error();
    return gs::dict_decode(dict, kind, codes, n, terms, lens);
}

GSMAT_API int gsmat_sparql_parse(const gsmat_dict *dict, const char *text, int64_t len, gsmat_sparql **out) {
    gs::clear_error();
    return gs::sparql_parse(dict, text, len, out);
}

GSMAT_API int gsmat_sparql_info(const gsmat_sparql *q, const gsmat_pattern **pats, int32_t *n_pats,
                                int32_t *n_vars, const int32_t **proj, int32_t *n_proj, int32_t *distinct) {
    gs::clear_error();
    return gs::sparql_info(q, pats, n_pats, n_vars, proj, n_proj, distinct);
}

GSMAT_API const char *gsmat_sparql_var_name(const gsmat_sparql *q, int32_t v) { return gs::sparql_var_name(q, v); }

GSMAT_API void gsmat_sparql_free(gsmat_sparql *q) { gs::sparql_free(q); }

GSMAT_API int gsmat_plan_cost(const gsmat_pattern *pats, int n_pats, int n_vars, const int64_t *keys,
                              const gsmat_pred_stats *stats, int32_t *order_out, int32_t *kinds_out,
                              double *est_out) {
    gs::clear_error();
    GS_TRY(gs::validate_bgp(pats, n_pats, n_vars));
    if (!keys || !stats || !order_out) return set_error(GSMAT_ERR_INVALID_ARG, "NULL argument");
    return gs::plan_bgp_cost(pats, n_pats, keys, stats, order_out, kinds_out, est_out);
}

GSMAT_API int gsmat_radix_sort_u64(uint64_t *d_keys, uint32_t *d_vals, int64_t n, int begin_bit, int end_bit,
                                   gsmat_stream_t stream) {
    gs::clear_error();
    if (n > 0 && !d_keys) return set_error(GSMAT_ERR_INVALID_ARG, "keys is NULL");
    return gs::radix_sort_u64(d_keys, d_vals, n, begin_bit, end_bit, (cudaStream_t)stream);
}

GSMAT_API int gsmat_sort_rows(const int32_t *const *d_cols, int V, int m, int bits, int64_t n,
                              int32_t *const *d_out, uint32_t flags, gsmat_stream_t stream) {
    gs::clear_error();
    if (flags > GSMAT_SORT_GATHER) return set_error(GSMAT_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
    if (V < 1 || V > gs::kMaxCols || !d_cols || !d_out) return set_error(GSMAT_ERR_INVALID_ARG, "bad columns");
    gs::Cols in;
    gs::OutCols out;
    for (int v = 0; v < gs::kMaxCols; ++v) {
        in.c[v] = v < V ? d_cols[v] : nullptr;
        out.c[v] = v < V ? d_out[v] : nullptr;
        if (v < V && n > 0 && (!in.c[v] || !out.c[v])) return set_error(GSMAT_ERR_INVALID_ARG, "column %d is NULL", v);
    }
    const int mode = flags == GSMAT_SORT_CARRY ? gs::kReorderCarry
                     : flags == GSMAT_SORT_GATHER ? gs::kReorderGather : gs::kReorderAuto;
    return gs::reorder_rows(in, V, m, bits, n, out, (cudaStream_t)stream, nullptr, mode);
}

GSMAT_API int gsmat_exclusive_scan_i32(const int32_t *d_in, int64_t *d_out, int64_t n, gsmat_stream_t stream) {
    gs::clear_error();
    return gs::exclusive_scan_i32(d_in, d_out, n, (cudaStream_t)stream, nullptr);
}

GSMAT_API int gsmat_exclusive_scan_i32_noalloc(const int32_t *d_in, int64_t *d_out, int64_t n,
                                               gsmat_stream_t stream) {
    gs::clear_error();
    return gs::exclusive_scan_i32_noalloc(d_in, d_out, n, (cudaStream_t)stream);
}

GSMAT_API int64_t gsmat_exclusive_scan_i32_noalloc_max(void) { return gs::exclusive_scan_i32_noalloc_max(); }

GSMAT_API int gsmat_store_set_tiles(gsmat_store *store, const gsmat_tiles *tiles) {
    gs::clear_error();
    if (!store || !tiles) return gs::set_error(GSMAT_ERR_INVALID_ARG, "NULL argument");
    gs::TileConfig tc;
    tc.expand_items = tiles->expand_items;
    tc.short_row = tiles->short_row;
    GS_TRY(gs::tile_config_check(tc));
    store->tiles = tc;
    return GSMAT_OK;
}

GSMAT_API int gsmat_store_get_tiles(const gsmat_store *store, gsmat_tiles *tiles) {
    gs::clear_error();
    if (!store || !tiles) return gs::set_error(GSMAT_ERR_INVALID_ARG, "NULL argument");
    tiles->expand_items = store->tiles.expand_items;
    tiles->short_row = store->tiles.short_row;
    return GSMAT_OK;
}

GSMAT_API int gsmat_store_tune(gsmat_store *store, const gsmat_bgp *bgps, int32_t n, gsmat_stream_t stream,
                               gsmat_tiles *best) {
    gs::clear_error();
    if (!best) return gs::set_error(GSMAT_ERR_INVALID_ARG, "best is NULL");
    gs::TileConfig tc;
    const int rc = gs::store_tune(store, bgps, n, (cudaStream_t)stream, &tc);
    gs::profile_flush();
    if (rc != GSMAT_OK) return rc;
    best->expand_items = tc.expand_items;
    best->short_row = tc.short_row;
    return GSMAT_OK;
}

GSMAT_API int gsmat_selftest_wait_expiry(int32_t poll_limit, gsmat_stream_t stream) {
    gs::clear_error();
    return gs::selftest_wait_expiry(poll_limit, (cudaStream_t)stream);
}

GSMAT_API int gsmat_profile_enable(int on) { return gs::profile_enable(on); }

GSMAT_API int64_t gsmat_launch_count(void) { return gs::launch_count(); }

GSMAT_API int gsmat_profile_read(gsmat_kernel_profile *out, int32_t cap, int32_t *n_out, int reset) {
    return gs::profile_read(out, cap, n_out, reset);
}

}  // extern "C"
