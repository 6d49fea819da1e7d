// Join kernels of one SM-based join step (Alg. 3) and their launchers.
#pragma once

#include "common.cuh"

namespace gs {

constexpr int kMaxCols = 32;

// Column set of a binding table (structure of arrays, int32 columns).
struct Cols {
    const int32_t *c[kMaxCols];
};
struct OutCols {
    int32_t *c[kMaxCols];
};

// A value that comes from a table column or is a constant.
struct ValueSrc {
    const int32_t *col;  // null -> constant
    int32_t constant;
    __device__ __forceinline__ int32_t at(int64_t i) const { return col ? col[i] : constant; }
};

// Count + exclusive scan (Alg. 4): for every input row i, N_i = size of the
// row of x_i on the given side of the predicate, first_i = its first entry;
// off[i] = sum of N_j for j < i, off[n] = total; *d_total = total.
int launch_count_scan(const StoreView &sv, int side, const PredSide &ps, const int32_t *x, int64_t n, int64_t *off,
                      int32_t *first, int64_t *d_total, int *err, cudaStream_t st);

// Gather-expand: output row j of [0, total) = parent row r (off[r] <= j <
// off[r+1]) with its k columns copied, plus the new column
// val[first_r + j - off[r]] appended as column k.
int launch_expand(const StoreView &sv, int side, const Cols &in, int k, int64_t n_in, const int64_t *off,
                  const int32_t *first, int64_t total, OutCols out, cudaStream_t st);

// Membership filter + compaction: keep row i iff (s_i, o_i) is an entry of
// the predicate (s_i, o_i from columns or constants); surviving rows' k
// columns are written in order to `out`; *d_count = survivors.
int launch_filter(const StoreView &sv, const PredSide &ps_s, const PredSide &ps_o, ValueSrc s, ValueSrc o,
                  const Cols &in, int k, int64_t n_in, OutCols out, int64_t *d_count, int *err, cudaStream_t st);

// Intersect-expand, count phase: counts[i] = |row(a_i) of predicate side
// (side_a, pa)  intersected with  row(b_i) of (side_b, pb)|.
int launch_isect_count(const StoreView &sv, int side_a, const PredSide &pa, ValueSrc a, int side_b, const PredSide &pb,
                       ValueSrc b, int64_t n, int32_t *counts, cudaStream_t st);
// Write phase: input row i's matches go to rows [off[i], off[i+1]) with the
// k input columns copied and the match appended as column k.
int launch_isect_write(const StoreView &sv, int side_a, const PredSide &pa, ValueSrc a, int side_b, const PredSide &pb,
                       ValueSrc b, int64_t n, const int64_t *off, const Cols &in, int k, int64_t total, OutCols out,
                       cudaStream_t st);

// Cartesian product: output row j = (input row j / m, relation row j % m);
// the relation has r_cols (1 or 2) columns of length m.
int launch_cross(const Cols &in, int k, int64_t n_in, const Cols &rel, int r_cols, int64_t m, OutCols out,
                 cudaStream_t st);

// Entries of one predicate (side 0) with key == val, as one column.
int launch_diag(const StoreView &sv, const PredSide &ps0, int32_t *out, int64_t *d_count, int *err, cudaStream_t st);

// Row ranges of constants: for request i, (first, last) of row x[i] of
// predicate slot ps[i] on side sd[i]; requests with slot < 0 give (0, 0).
int launch_const_lookup(const StoreView &sv, const PredSide *d_sides, int n_pred, const int32_t *d_req, int n_req,
                        int32_t *d_out, cudaStream_t st);

// keys[i] = columns cols[0..nc) of row perm[i] (or row i if perm is null)
// packed most-significant first with `bits` bits each.
// Stable reorder of an n-row table (cols = its V columns in variable order)
// by variables 0..m-1, lexicographically, into out (V columns).  Keys pack
// the variables `bits` bits each, as many per 64-bit key as fit; wider
// orders sort chunk by chunk, least significant first.  *err_word is set if a
// bounded wait expired (may be null).
// mode: how the non-key columns reach the output when both ways apply
// (they fit one 64-bit payload, one key chunk, more than 2048 rows):
// carried through the passes, gathered after the sort, or chosen by size.
enum { kReorderAuto = 0, kReorderCarry = 1, kReorderGather = 2 };
int reorder_rows(const Cols &cols, int V, int m, int bits, int64_t n, const OutCols &out, cudaStream_t st,
                 int *err_word, int mode = kReorderAuto);
// dst[i * k + c] = in[c][i] (row-major interleave).
int launch_interleave(const Cols &in, int k, int64_t n, int32_t *dst, cudaStream_t st);
// out[c][i] = in[c][i] (copy k columns).
int launch_copy_cols(const Cols &in, int k, int64_t n, OutCols out, cudaStream_t st);

}  // namespace gs
