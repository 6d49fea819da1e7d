// Single-pass stable selection ("prefix-sum compaction") over an index
// range: every tile evaluates a predicate per index, ranks its hits with a
// block scan, obtains the number of hits of all earlier tiles by decoupled
// look-back and lets the operator write each hit at its final position.
// Output order equals input order, so results are deterministic.
#pragma once

#include "common.cuh"

namespace gs {

// Op must provide:
//   __device__ bool flag(int64_t i) const;          // keep index i?
//   __device__ void emit(int64_t i, int64_t j) const; // write hit i at output j
template <int BLOCK, int ITEMS, class Op>
__global__ void __launch_bounds__(BLOCK) select_kernel(Op op, int64_t n, LookbackScratch ls, int64_t *d_count) {
    __shared__ int tile_sm;
    __shared__ int64_t scan_sm[BLOCK / 32 + 1];
    __shared__ int64_t prefix_sm;
    const int tile = acquire_tile_id(ls, &tile_sm);
    const int64_t i0 = (int64_t)tile * (BLOCK * ITEMS) + (int64_t)threadIdx.x * ITEMS;
    bool f[ITEMS];
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int64_t i = i0 + j;
        f[j] = (i < n) && op.flag(i);
        cnt += f[j] ? 1 : 0;
    }
    int64_t tot;
    const int64_t ex = block_exclusive_sum<BLOCK>(cnt, scan_sm, &tot);
    const int64_t pre = tile_lookback(ls, tile, tot, &prefix_sm);
    int64_t out = pre + ex;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        if (f[j]) op.emit(i0 + j, out++);
    }
    if (tile == (int)gridDim.x - 1 && threadIdx.x == 0) *d_count = pre + tot;
}

// Launch select_kernel over [0, n); *d_count receives the number of hits.
// A bounded wait that expires sets *err_word (device int) when given.
template <class Op, int BLOCK = 256, int ITEMS = 4>
int run_select(const Op &op, int64_t n, int64_t *d_count, cudaStream_t st, int *err_word) {
    if (n <= 0) {
        GS_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int64_t), st));
        return GSMAT_OK;
    }
    constexpr int TILE = BLOCK * ITEMS;
    const int64_t ntiles = (n + TILE - 1) / TILE;
    if (ntiles > INT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "selection over %lld items", (long long)n);
    LookbackBuf lb;
    GS_TRY(lb.make(ntiles, st, err_word));
    select_kernel<BLOCK, ITEMS, Op><<<(unsigned)ntiles, BLOCK, 0, st>>>(op, n, lb.view, d_count);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

}  // namespace gs
