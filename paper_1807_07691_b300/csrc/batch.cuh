// Device-side program of a batch of BGPs and the persistent kernel's
// arguments (see batch.cu).
#pragma once

#include "common.cuh"

namespace gs {

// One plan step, with every operand resolved to a column of the running
// table (or a constant) on the host.
struct BStep {
    int32_t kind;      // GSMAT_STEP_*
    int32_t slot;      // predicate slot in the store
    int32_t s_col;     // column holding the subject, -1 when constant or new
    int32_t o_col;     // column holding the object, -1 when constant or new
    int32_t s_const;   // subject constant (when s_col < 0 and the subject is known)
    int32_t o_const;
    int32_t diag;      // CROSS of ?x p ?x
    int32_t c_first;   // EXPAND from a constant: entry range of its row
    int32_t c_last;
    int32_t swap;      // CROSS of M_p: take it by object, columns (o, s)
    // GSMAT_STEP_INTERSECT: an EXPAND from a bound variable whose new
    // variable a later FILTER ties to a variable bound before it (or a
    // constant); that FILTER's step has kind GSMAT_STEP_FUSED.
    int32_t a_side;    // side of the EXPAND's row (0: by subject, 1: by object)
    int32_t f_slot;    // the filter's predicate slot
    int32_t f_side;    // side of the filter's row (1 when the new variable is its subject)
    int32_t b_col;     // column of the filter's other end (-1: the constant b_const)
    int32_t b_const;
};

struct BQuery {
    int32_t step0;     // first step in the step array
    int32_t n_steps;
    int32_t n_vars;
    int32_t m_sort;    // leading variables to sort for variable order (0: none)
    int32_t absent;    // a predicate is missing: empty result
    int32_t _pad;
    int32_t col_of_var[32];  // final plan column of each variable
};

enum { BR_OK = 0, BR_OVERFLOW = 1, BR_NEEDS_SORT = 2 };

struct BResult {
    int64_t rows;
    int32_t status;
    int32_t ncols;
    const int32_t *col[32];  // per variable
};

struct BatchArgs {
    StoreView sv;
    const PredSide *sides;   // [2][n_pred]
    int n_pred;
    int bits;                // bits per packed variable in the sort key
    const BStep *steps;
    const BQuery *queries;
    int n_queries;
    BResult *results;
    char *arena;
    unsigned long long *arena_top;
    unsigned long long arena_cap;
    unsigned int *queue_head;
    int64_t max_rows;        // per table; larger tables send the query to the plain path
};

// expand_slots: output slots per thread per round of the expand loop (1 or 4)
int launch_batch_kernel(const BatchArgs &a, int block, int expand_slots, int grid, cudaStream_t st);

// Host resources a batch may borrow instead of creating its own (a server
// keeps one set per in-flight slot and reuses it): a stream, four events and
// pinned buffers for up to `cap` result descriptors and the two control
// words.
struct BatchResources {
    cudaStream_t st;
    cudaEvent_t ev[4];
    BResult *results_host;
    unsigned long long *ctrl_host;
    int cap;
};

// One result table of a segmented reorder: its rows are rows
// [row_off, row_off + rows) of the concatenation; col[v] = the column of
// variable v (variables 0..m-1 are the sort key); out = V columns of rows.
// On the device an array of n_segs descriptors is followed by the int64
// array of their row_off values (see upload_segs), which the kernels
// search.
struct SegDesc {
    int64_t row_off;
    int64_t rows;
    int32_t m;
    int32_t V;
    const int32_t *col[32];
    int32_t *out;
};
// keys[g] = the variables [vb, ve) of the row at source position src (g, or
// perm_in[g]) packed `bits` each, with the segment index at seg_shift when
// seg_shift >= 0; idx_bits > 0 appends src in the low idx_bits bits (and
// perm_out is not written), else perm_out[g] = g when perm_in is null.
int launch_seg_pack(const SegDesc *segs, int n_segs, int bits, int vb, int ve, int seg_shift, int idx_bits,
                    const uint32_t *perm_in, int64_t total, uint64_t *keys, uint32_t *perm_out, cudaStream_t st);
// Carried columns of a segmented reorder: keys = (segment << kb) | the
// variables [0, m); pay = the segment's variables [m, V); and back into each
// segment's out after the sort.
int launch_seg_pack_wide(const SegDesc *segs, int n_segs, int bits, int m, int kb, int64_t total, uint64_t *keys,
                         uint64_t *pay, cudaStream_t st);
int launch_seg_unpack_wide(const SegDesc *segs, int n_segs, int bits, int m, int64_t total, const uint64_t *keys,
                           const uint64_t *pay, cudaStream_t st);
// perm[g] = the low idx_bits bits of keys[g].
int launch_key_low_bits(const uint64_t *keys, int idx_bits, int64_t total, uint32_t *perm, cudaStream_t st);
// out rows of every segment from the rows perm[p] (a plain copy when perm
// is null).
int launch_seg_gather(const SegDesc *segs, int n_segs, int64_t total, const uint32_t *perm, cudaStream_t st);

}  // namespace gs
