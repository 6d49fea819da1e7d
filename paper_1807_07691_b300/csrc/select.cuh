// Single-pass stable selection ("prefix-sum compaction") over an index
// range: every tile evaluates a predicate per index, ranks its hits with a
// block scan, obtains the number of hits of all earlier tiles by decoupled
// look-back and lets the operator write each hit at its final position.
// Output order equals input order, so results are deterministic.
#pragma once

#include "common.cuh"

#ifndef GSMAT_SELECT_ITEMS
#define GSMAT_SELECT_ITEMS 8  // indices per thread and tile
#endif

namespace gs {

// Op must provide:
//   __device__ bool flag(int64_t i) const;          // keep index i?
//   __device__ void emit(int64_t i, int64_t j) const; // write hit i at output j
// and may provide
//   __device__ void visit(int64_t i) const;         // called once for every i < n
template <class Op>
__device__ __forceinline__ auto select_visit(const Op &op, int64_t i, int) -> decltype(op.visit(i), void()) {
    op.visit(i);
}
template <class Op>
__device__ __forceinline__ void select_visit(const Op &, int64_t, long) {}

template <int BLOCK, int ITEMS, class Op>
__global__ void __launch_bounds__(BLOCK) select_kernel(Op op, int64_t n, LookbackScratch ls, int64_t *d_count) {
    constexpr int W = BLOCK / 32;
    __shared__ int tile_sm;
    __shared__ int64_t prefix_sm;
    __shared__ int wsum[W + 1];
    const int tile = acquire_tile_id(ls, &tile_sm);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // warp-striped: warp w takes 32 * ITEMS consecutive indices, lane l the
    // l-th of every 32, so reads and the compacted writes are coalesced
    const int64_t wbase = (int64_t)tile * (BLOCK * ITEMS) + (int64_t)warp * (32 * ITEMS);
    // all predicates first (their loads in flight together), then the votes
    bool f[ITEMS];
    if (wbase + 32 * ITEMS <= n) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) f[j] = op.flag(wbase + j * 32 + lane);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) select_visit(op, wbase + j * 32 + lane, 0);
    } else {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int64_t i = wbase + j * 32 + lane;
            f[j] = i < n && op.flag(i);
            if (i < n) select_visit(op, i, 0);
        }
    }
    unsigned hit[ITEMS];
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        hit[j] = __ballot_sync(0xffffffffu, f[j]);
        cnt += __popc(hit[j]);
    }
    if (lane == 0) wsum[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        const int c = lane < W ? wsum[lane] : 0;
        int inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane < W) wsum[lane] = inc - c;
        if (lane == W - 1) wsum[W] = inc;
    }
    __syncthreads();
    const int64_t tot = wsum[W];
    const int64_t pre = tile_lookback(ls, tile, tot, &prefix_sm);
    int64_t out = pre + wsum[warp];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        if ((hit[j] >> lane) & 1u) op.emit(wbase + j * 32 + lane, out + __popc(hit[j] & lt));
        out += __popc(hit[j]);
    }
    if (tile == (int)gridDim.x - 1 && threadIdx.x == 0) *d_count = pre + tot;
}

// Two nested selections in one pass.  Op provides
//   __device__ void flags(int64_t i, bool &f1, bool &f2) const;  // f2 implies f1
//   __device__ void emit(int64_t i, int64_t j1, int64_t j2) const;  // j2 = -1 unless f2
// where j1 ranks i among the f1 hits and j2 among the f2 hits.  Both counts
// travel in one look-back word (31 bits each, so n < 2^31); d_count[0] and
// d_count[1] receive the totals.
template <int BLOCK, int ITEMS, class Op>
__global__ void __launch_bounds__(BLOCK) select2_kernel(Op op, int64_t n, LookbackScratch ls, int64_t *d_count) {
    constexpr int W = BLOCK / 32;
    __shared__ int tile_sm;
    __shared__ int64_t prefix_sm;
    __shared__ int wsum[2][W + 1];
    const int tile = acquire_tile_id(ls, &tile_sm);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wbase = (int64_t)tile * (BLOCK * ITEMS) + (int64_t)warp * (32 * ITEMS);
    bool f1[ITEMS], f2[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        f1[j] = f2[j] = false;
        if (i < n) op.flags(i, f1[j], f2[j]);
    }
    unsigned h1[ITEMS], h2[ITEMS];
    int c1 = 0, c2 = 0;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        h1[j] = __ballot_sync(0xffffffffu, f1[j]);
        h2[j] = __ballot_sync(0xffffffffu, f2[j]);
        c1 += __popc(h1[j]);
        c2 += __popc(h2[j]);
    }
    if (lane == 0) {
        wsum[0][warp] = c1;
        wsum[1][warp] = c2;
    }
    __syncthreads();
    if (warp < 2) {
        const int c = lane < W ? wsum[warp][lane] : 0;
        int inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane < W) wsum[warp][lane] = inc - c;
        if (lane == W - 1) wsum[warp][W] = inc;
    }
    __syncthreads();
    const int64_t t1 = wsum[0][W], t2 = wsum[1][W];
    const int64_t pre = tile_lookback(ls, tile, t1 | (t2 << 31), &prefix_sm);
    const int64_t p1 = pre & ((int64_t(1) << 31) - 1), p2 = pre >> 31;
    int64_t o1 = p1 + wsum[0][warp], o2 = p2 + wsum[1][warp];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        if ((h1[j] >> lane) & 1u) {
            op.emit(wbase + j * 32 + lane, o1 + __popc(h1[j] & lt),
                    ((h2[j] >> lane) & 1u) ? o2 + __popc(h2[j] & lt) : int64_t(-1));
        }
        o1 += __popc(h1[j]);
        o2 += __popc(h2[j]);
    }
    if (tile == (int)gridDim.x - 1 && threadIdx.x == 0) {
        d_count[0] = p1 + t1;
        d_count[1] = p2 + t2;
    }
}

template <class Op, int BLOCK = 256, int ITEMS = GSMAT_SELECT_ITEMS>
int run_select2(const Op &op, int64_t n, int64_t *d_count, cudaStream_t st, int *err_word) {
    if (n <= 0) {
        GS_CUDA(cudaMemsetAsync(d_count, 0, 2 * sizeof(int64_t), st));
        return GSMAT_OK;
    }
    if (n >= (int64_t(1) << 31)) return set_error(GSMAT_ERR_CAPACITY, "two-count selection over %lld items", (long long)n);
    constexpr int TILE = BLOCK * ITEMS;
    const int64_t ntiles = (n + TILE - 1) / TILE;
    LookbackBuf lb;
    GS_TRY(lb.make(ntiles, st, err_word));
    select2_kernel<BLOCK, ITEMS, Op><<<(unsigned)ntiles, BLOCK, 0, st>>>(op, n, lb.view, d_count);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

// Launch select_kernel over [0, n); *d_count receives the number of hits.
// A bounded wait that expires sets *err_word (device int) when given.
template <class Op, int BLOCK = 256, int ITEMS = GSMAT_SELECT_ITEMS>
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
