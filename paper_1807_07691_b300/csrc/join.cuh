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

// Tile shapes of the plain path's join kernels, chosen per store (by
// gsmat_store_tune or gsmat_store_set_tiles): output slots plus parent rows
// per CTA of the expand and product kernels (their merge-path pieces), and
// the row length up to which the membership filter searches the subject's
// row directly instead of looking at the object's row as well.
struct TileConfig {
    int expand_items = 2048;  // 512, 1024, 2048, 4096 or 8192
    int short_row = 64;       // 1 .. 4096
};
int tile_config_check(const TileConfig &tc);

// A value that comes from a table column or is a constant.
struct ValueSrc {
    const int32_t *col;  // null -> constant
    int32_t constant;
    __device__ __forceinline__ int32_t at(int64_t i) const { return col ? col[i] : constant; }
};

// Intersection of two sorted entry lists by one warp (all 32 lanes call it
// with the same arguments): the row of a_val on predicate side (sa, pa) and
// the row of b_val on (sb, pb).  The warp walks the shorter list in chunks of
// 32; each lane binary-searches its element in the part of the longer list
// not yet passed, and ballot / popc rank the matches.  emit(r, v) is called
// by the lane holding the r-th match (ascending) v; returns the count in
// every lane.  A new variable bound by two patterns of Alg. 3 takes exactly
// these values, in the order an expand followed by a filter gives.
template <class Emit>
__device__ __forceinline__ int warp_intersect(const SideView &sa, const PredSide &pa, int32_t a_val,
                                              const SideView &sb, const PredSide &pb, int32_t b_val, Emit emit) {
    const int lane = threadIdx.x & 31;
    const int2 ra = row_range(sa, pa, a_val);
    const int2 rb = row_range(sb, pb, b_val);
    const int la = ra.y - ra.x, lb = rb.y - rb.x;
    if (la <= 0 || lb <= 0) return 0;
    const int32_t *S = la <= lb ? sa.val + ra.x : sb.val + rb.x;
    const int32_t *L = la <= lb ? sb.val + rb.x : sa.val + ra.x;
    const int ls = la <= lb ? la : lb, ll = la <= lb ? lb : la;
    int count = 0;
    int lo_all = 0;  // no element of L before this position can match any later element of S
    for (int base = 0; base < ls; base += 32) {
        const int idx = base + lane;
        int32_t v = 0;
        bool found = false;
        int pos = ll;
        if (idx < ls) {
            v = __ldg(S + idx);
            int lo = lo_all, hi = ll;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(L + mid) < v) lo = mid + 1; else hi = mid;
            }
            pos = lo;
            found = lo < ll && __ldg(L + lo) == v;
        }
        const unsigned m = __ballot_sync(0xffffffffu, found);
        if (found) emit(count + __popc(m & ((1u << lane) - 1u)), v);
        count += __popc(m);
        // the chunk's last element bounds the next chunk's searches from below
        const int last = min(31, ls - 1 - base);
        lo_all = __shfl_sync(0xffffffffu, pos, last);
        if (lo_all >= ll) break;
    }
    return count;
}

// Count + exclusive scan (Alg. 4): for every input row i, N_i = size of the
// row of x_i on the given side of the predicate, first_i = its first entry;
// off[i] = sum of N_j for j < i, off[n] = total; *d_total = total.
int launch_count_scan(const StoreView &sv, int side, const PredSide &ps, const int32_t *x, int64_t n, int64_t *off,
                      int32_t *first, int64_t *d_total, int *err, cudaStream_t st);

// Gather-expand: output row j of [0, total) = parent row r (off[r] <= j <
// off[r+1]) with its k columns copied, plus the new column
// val[first_r + j - off[r]] appended as column k.
int launch_expand(const StoreView &sv, int side, const Cols &in, int k, int64_t n_in, const int64_t *off,
                  const int32_t *first, int64_t total, OutCols out, cudaStream_t st,
                  const TileConfig &tc = TileConfig());

// Membership filter + compaction: keep row i iff (s_i, o_i) is an entry of
// the predicate (s_i, o_i from columns or constants); surviving rows' k
// columns are written in order to `out`; *d_count = survivors.
int launch_filter(const StoreView &sv, const PredSide &ps_s, const PredSide &ps_o, ValueSrc s, ValueSrc o,
                  const Cols &in, int k, int64_t n_in, OutCols out, int64_t *d_count, int *err, cudaStream_t st,
                  const TileConfig &tc = TileConfig());

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

// ---------------------------------------------------------------------------
// Product of independent expansions.  When the last steps of a plan each
// bind one new variable from a list that depends only on the table before
// them -- the row of a bound column's value (EXPAND from a variable), a
// constant's row (EXPAND from a constant) or a whole matrix (CROSS, two new
// variables) -- every input row r joins with the Cartesian product of its
// lists L_1(r) x ... x L_F(r) (Alg. 3 applied step by step gives exactly
// these rows).  The product is written in one pass, nested in a chosen
// factor order (outermost first), each list ascending, so that output rows
// ascend in (input columns, factor columns in nesting order).

// Division by a divisor that is fixed for many dividends: the multiply and
// shift of Granlund and Montgomery ("Division by invariant integers using
// multiplication", PLDI 1994), round-up form: for 1 <= d < 2^32 let
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1 (< 2^32); then for
// every 32-bit n, n / d = (mulhi(n, m) + n) >> l, the sum taken in 64 bits.
struct FastDiv {
    uint32_t d;
    uint32_t m;
    uint32_t l;
};
__host__ __device__ inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    uint32_t l = 0;
    while (l < 32 && (uint64_t(1) << l) < (uint64_t)d) ++l;
    f.l = l;
    f.m = d == 0 ? 0u : (uint32_t)((((uint64_t(1) << l) - (uint64_t)d) << 32) / (uint64_t)d + 1);
    return f;
}
__host__ __device__ inline uint32_t fastdiv_quot(uint32_t n, const FastDiv &f) {
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(n, f.m);
#else
    const uint32_t t = (uint32_t)(((uint64_t)n * (uint64_t)f.m) >> 32);
#endif
    return (uint32_t)(((uint64_t)t + (uint64_t)n) >> f.l);
}

constexpr int kMaxProdFactors = 16;
enum { kProdRow = 0, kProdList = 1, kProdPairs = 2 };

struct ProdFactor {
    int kind;          // kProdRow, kProdList or kProdPairs
    int side;          // kProdRow: store side whose row is taken
    int xcol;          // kProdRow: input column holding the row's id
    int slot;          // kProdRow: index among the row factors (first / len arrays)
    PredSide ps;       // kProdRow: the predicate side
    const int32_t *a;  // kProdList: the values; kProdPairs: first column
    const int32_t *b;  // kProdPairs: second column
    uint32_t len;      // kProdList / kProdPairs: length
    FastDiv div;       // kProdList / kProdPairs: divisor len
    FastDiv inner;     // fixed products only: divisor = product of the inner factors' lengths
    int out0;          // output column of the factor's (first) value
};
struct ProdSpec {
    int nf;    // factors, outermost first
    int nrow;  // factors of kind kProdRow (slots 0..nrow-1)
    ProdFactor f[kMaxProdFactors];
};

// Count + scan: N_r = product over the factors of |L_i(r)| (saturating at
// 2^32; a total past 2^32 - 1 rows is refused by the caller);
// off[r] = exclusive prefix, off[n] = *d_total = total; for row factor with
// slot s: first[s * n + r] / len[s * n + r] = its row's entry range.
int launch_product_count_scan(const StoreView &sv, const ProdSpec &spec, const Cols &in, int64_t n, int64_t *off,
                              int32_t *first, int32_t *len, int64_t *d_total, int *err, cudaStream_t st);
// Write: output row j of [0, total) belongs to input row r (off[r] <= j <
// off[r+1]); its k input columns are copied and q = j - off[r] is split in
// mixed radix over the factors (innermost factor fastest) to pick each
// factor's entry.
int launch_product(const StoreView &sv, const ProdSpec &spec, const Cols &in, int k, int64_t n_in, const int64_t *off,
                   const int32_t *first, const int32_t *len, int64_t total, OutCols out, cudaStream_t st,
                  const TileConfig &tc = TileConfig());
// The product of fixed lists only (no input columns, one input row):
// total = product of the factors' lengths (< 2^32).
int launch_product_fixed(const ProdSpec &spec, int64_t total, OutCols out, cudaStream_t st);

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
