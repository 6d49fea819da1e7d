// Result tables and the query entry points shared with the C ABI layer.
#pragma once

#include "common.cuh"
#include "join.cuh"

struct gsmat_table {
    int64_t rows = 0;
    int32_t ncols = 0;
    int32_t vars[32] = {0};
    const int32_t *col[32] = {nullptr};
    gs::DevBuf storage;  // owns the columns
    gsmat_query_stats stats{};
    int32_t id_bits = 31;  // every value is below 2^id_bits
};

namespace gs {

// shard / n_shards: evaluate only what derives from the shard-th of n_shards
// contiguous parts of the first plan step's relation.
int query_run(const gsmat_store *S, const gsmat_pattern *pats, int n_pats, int n_vars, uint32_t flags, cudaStream_t st,
              gsmat_table **out, int shard = 0, int n_shards = 1);
// Rows of k tables with the same columns, together, ascending (gsmat_table_merge).
int table_merge(const gsmat_table *const *tables, int k, cudaStream_t st, gsmat_table **out);
// sync = false: enqueue only (the caller keeps T alive until st passes it).
int table_copy(const gsmat_table *T, int32_t *dst, int dst_on_device, cudaStream_t st, bool sync = true);
// Reorder a table given in plan column order (rows ascending in that order)
// to variable order, rows ascending; the result owns its columns.
int reorder_view(const gsmat_store *S, const int32_t *const *plan_cols, const int32_t *plan_vars, int V, int64_t rows,
                 cudaStream_t st, gsmat_table **out);
// Time the BGPs under every candidate tile shape and keep the fastest on the
// store (gsmat_store_tune).
int store_tune(gsmat_store *S, const gsmat_bgp *bgps, int32_t n, cudaStream_t st, TileConfig *best);
// Projection / DISTINCT of a table (gsmat_table_project).
int table_project(const gsmat_table *T, const int32_t *vars, int32_t n, int distinct, cudaStream_t st,
                  gsmat_table **out);
// Columns of a table in the order the plan binds variables, and the number
// of leading variables a stable reorder must sort (see canonical_order).
int leading_sort_vars(const int32_t *plan_vars, int V);

}  // namespace gs
