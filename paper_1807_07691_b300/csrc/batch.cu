// Batched BGP evaluation: many queries in one persistent kernel.
//
// The plain path (query.cu) runs one query at a time and synchronises with
// the host once per join step; for small queries that latency, not the
// data, dominates.  Here the host plans every query of a batch (Alg. 1),
// encodes each plan as a short step program and uploads all programs at
// once; a persistent kernel then pulls query ids from a device work queue
// (an atomic counter) and each CTA executes one query's joins (Alg. 2 and
// 3, the count / offset / write structure of Alg. 4) with CTA-wide loops,
// allocating its tables from a device arena with a bump pointer.  No host
// round trip happens inside the batch.  A query that would exceed the
// arena or the per-query row cap is marked and re-run on the plain path;
// a result that needs a reorder larger than the shared-memory sort is
// finished by the multi-CTA reorder.  Results are identical to the plain
// path's.
//
// The launch sequence (queue/arena reset, persistent kernel, result copy)
// is captured once per prepared batch as a CUDA graph and replayed.
#include <string.h>

#include <algorithm>
#include <vector>

#include "batch.cuh"
#include "join.cuh"
#include "plan.h"
#include "query.cuh"
#include "store.cuh"

namespace gs {

namespace {

constexpr int kSmemSortRows = 2048;

__device__ __forceinline__ bool member(const SideView &s0, const SideView &s1, const PredSide &p0, const PredSide &p1,
                                       int32_t x, int32_t y) {
    const int2 a = row_range(s0, p0, x);
    const int la = a.y - a.x;
    if (la <= 0) return false;
    if (la <= 64) return sorted_contains(s0.val, a.x, a.y, y);
    const int2 b = row_range(s1, p1, y);
    const int lb = b.y - b.x;
    if (lb <= 0) return false;
    if (la <= lb) return sorted_contains(s0.val, a.x, a.y, y);
    return sorted_contains(s1.val, b.x, b.y, x);
}

template <int BLOCK>
struct CtaShared {
    const int32_t *col[kMaxCols];
    const int32_t *ncol[kMaxCols];
    int64_t rows;
    int64_t scan[BLOCK / 32 + 1];
    unsigned long long alloc_off;
    int q;
    int ncols;
    int status;
    unsigned long long skey[kSmemSortRows];
    uint16_t sidx[kSmemSortRows];
};

template <int BLOCK>
__device__ __forceinline__ int32_t *cta_alloc(const BatchArgs &a, CtaShared<BLOCK> &sm, size_t bytes) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long b = (bytes + 255) & ~255ull;
        const unsigned long long off = atomicAdd(a.arena_top, b);
        sm.alloc_off = (off + b <= a.arena_cap) ? off : ~0ull;
    }
    __syncthreads();
    const unsigned long long off = sm.alloc_off;
    return off == ~0ull ? nullptr : reinterpret_cast<int32_t *>(a.arena + off);
}

// Exclusive block sum of v; *total gets the block total.
template <int BLOCK>
__device__ __forceinline__ int64_t cta_scan(CtaShared<BLOCK> &sm, int64_t v, int64_t *total) {
    return block_exclusive_sum<BLOCK>(v, sm.scan, total);
}

// EPT: output slots per thread per round of the expand loop (a tile shape
// the autotuner picks): one search per EPT consecutive slots, the next
// parents found by stepping forward.
template <int BLOCK, int EPT>
__device__ void run_query(const BatchArgs &a, CtaShared<BLOCK> &sm, int q) {
    const BQuery &Q = a.queries[q];
    const int tid = threadIdx.x;
    if (tid == 0) {
        sm.rows = Q.absent ? 0 : 1;
        sm.ncols = 0;
        sm.status = BR_OK;
    }
    __syncthreads();
    for (int si = 0; si < Q.n_steps; ++si) {
        if (sm.rows == 0 || sm.status != BR_OK) break;
        const BStep &S = a.steps[Q.step0 + si];
        const PredSide p0 = a.sides[S.slot];
        const PredSide p1 = a.sides[a.n_pred + S.slot];
        const int64_t n = sm.rows;
        const int k = sm.ncols;
        const bool unit = (n == 1 && k == 0);
        if (S.kind == GSMAT_STEP_FUSED) continue;  // applied by the INTERSECT before it
        if (S.kind == GSMAT_STEP_INTERSECT) {
            // count the intersections (a warp per row), offsets by a running
            // CTA scan, then each warp writes its rows' matches
            const PredSide pa = S.a_side == 0 ? p0 : p1;
            const PredSide pb = a.sides[S.f_side * a.n_pred + S.f_slot];
            const SideView &sva = a.sv.side[S.a_side];
            const SideView &svb = a.sv.side[S.f_side];
            const int32_t *x = sm.col[S.a_side == 0 ? S.s_col : S.o_col];
            const int32_t *bc = S.b_col >= 0 ? sm.col[S.b_col] : nullptr;
            int32_t *tmp = cta_alloc(a, sm, sizeof(int32_t) * (size_t)(2 * n + 2));
            if (!tmp) {
                if (tid == 0) sm.status = BR_OVERFLOW;
                __syncthreads();
                break;
            }
            int32_t *cnt = tmp;      // n
            int32_t *off = tmp + n;  // n + 1
            const int warp = tid >> 5;
            constexpr int kWarps = BLOCK / 32;
            for (int64_t i = warp; i < n; i += kWarps) {
                const int c = warp_intersect(sva, pa, x[i], svb, pb, bc ? bc[i] : S.b_const, [](int, int32_t) {});
                if ((tid & 31) == 0) cnt[i] = c;
            }
            __syncthreads();
            int64_t carry = 0;
            for (int64_t base = 0; base < n; base += BLOCK) {
                const int64_t i = base + tid;
                const int c = i < n ? cnt[i] : 0;
                int64_t tot;
                const int64_t ex = cta_scan(sm, c, &tot);
                if (i < n && carry + ex <= a.max_rows) off[i] = (int32_t)(carry + ex);
                carry += tot;
                if (carry > a.max_rows) break;  // uniform
            }
            if (carry > a.max_rows) {
                if (tid == 0) sm.status = BR_OVERFLOW;
                __syncthreads();
                break;
            }
            if (tid == 0) off[n] = (int32_t)carry;
            const int64_t total = carry;
            int32_t *out = total > 0 ? cta_alloc(a, sm, sizeof(int32_t) * (size_t)total * (k + 1)) : nullptr;
            if (total > 0 && !out) {
                if (tid == 0) sm.status = BR_OVERFLOW;
                __syncthreads();
                break;
            }
            __syncthreads();
            for (int64_t i = warp; i < n; i += kWarps) {
                const int64_t o0 = off[i];
                if (off[i + 1] == o0) continue;  // warp-uniform
                warp_intersect(sva, pa, x[i], svb, pb, bc ? bc[i] : S.b_const, [&](int r, int32_t v) {
                    const int64_t j = o0 + r;
                    for (int c = 0; c < k; ++c) out[(size_t)c * total + j] = sm.col[c][i];
                    out[(size_t)k * total + j] = v;
                });
            }
            __syncthreads();
            if (tid == 0) {
                for (int c = 0; c <= k; ++c) sm.col[c] = out + (size_t)c * total;
                sm.ncols = k + 1;
                sm.rows = total;
            }
            __syncthreads();
            continue;
        }
        if (S.kind == GSMAT_STEP_FILTER) {
            int32_t *out = k > 0 ? cta_alloc(a, sm, sizeof(int32_t) * (size_t)n * k) : nullptr;
            if (k > 0 && !out) {
                if (tid == 0) sm.status = BR_OVERFLOW;
                __syncthreads();
                break;
            }
            int64_t carry = 0;
            for (int64_t base = 0; base < n; base += BLOCK) {
                const int64_t i = base + tid;
                bool f = false;
                if (i < n) {
                    const int32_t x = S.s_col >= 0 ? sm.col[S.s_col][i] : S.s_const;
                    const int32_t y = S.o_col >= 0 ? sm.col[S.o_col][i] : S.o_const;
                    f = member(a.sv.side[0], a.sv.side[1], p0, p1, x, y);
                }
                int64_t tot;
                const int64_t ex = cta_scan(sm, f ? 1 : 0, &tot);
                if (f) {
                    for (int c = 0; c < k; ++c) out[(size_t)c * n + carry + ex] = sm.col[c][i];
                }
                carry += tot;
            }
            __syncthreads();
            if (tid == 0) {
                for (int c = 0; c < k; ++c) sm.col[c] = out + (size_t)c * n;
                sm.rows = carry;
            }
            __syncthreads();
        } else if ((S.kind == GSMAT_STEP_EXPAND_S || S.kind == GSMAT_STEP_EXPAND_O) &&
                   (S.kind == GSMAT_STEP_EXPAND_S ? S.s_col : S.o_col) >= 0) {
            const int side = S.kind == GSMAT_STEP_EXPAND_S ? 0 : 1;
            const SideView &sv = a.sv.side[side];
            const PredSide &ps = side == 0 ? p0 : p1;
            const int32_t *x = sm.col[side == 0 ? S.s_col : S.o_col];
            // count + offsets (Alg. 4: N, then P by a running scan)
            int32_t *tmp = cta_alloc(a, sm, sizeof(int32_t) * (size_t)(2 * n + 2));
            if (!tmp) {
                if (tid == 0) sm.status = BR_OVERFLOW;
                __syncthreads();
                break;
            }
            int32_t *off = tmp;             // n + 1
            int32_t *fst = tmp + n + 1;     // n
            int64_t carry = 0;
            for (int64_t base = 0; base < n; base += BLOCK) {
                const int64_t i = base + tid;
                int cnt = 0, f0 = 0;
                if (i < n) {
                    const int2 r = row_range(sv, ps, x[i]);
                    cnt = r.y - r.x;
                    f0 = r.x;
                }
                int64_t tot;
                const int64_t ex = cta_scan(sm, cnt, &tot);
                if (i < n && carry + ex <= a.max_rows) {
                    off[i] = (int32_t)(carry + ex);
                    fst[i] = f0;
                }
                carry += tot;
                if (carry > a.max_rows) break;  // uniform: carry is the same in every thread
            }
            if (carry > a.max_rows) {
                if (tid == 0) sm.status = BR_OVERFLOW;
                __syncthreads();
                break;
            }
            if (tid == 0) off[n] = (int32_t)carry;
            const int64_t total = carry;
            int32_t *out = total > 0 ? cta_alloc(a, sm, sizeof(int32_t) * (size_t)total * (k + 1)) : nullptr;
            if (total > 0 && !out) {
                if (tid == 0) sm.status = BR_OVERFLOW;
                __syncthreads();
                break;
            }
            __syncthreads();
            const int32_t *val = sv.val;
            for (int64_t jg = (int64_t)tid * EPT; jg < total; jg += (int64_t)BLOCK * EPT) {
                // parent of jg: largest r with off[r] <= jg
                int64_t lo = 0, hi = n - 1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) >> 1;
                    if (off[mid] <= jg) lo = mid; else hi = mid - 1;
                }
#pragma unroll
                for (int t = 0; t < EPT; ++t) {
                    const int64_t j = jg + t;
                    if (j >= total) break;
                    while (lo + 1 < n && off[lo + 1] <= j) ++lo;
                    for (int c = 0; c < k; ++c) out[(size_t)c * total + j] = sm.col[c][lo];
                    out[(size_t)k * total + j] = val[fst[lo] + (j - off[lo])];
                }
            }
            __syncthreads();
            if (tid == 0) {
                for (int c = 0; c <= k; ++c) sm.col[c] = out + (size_t)c * total;
                sm.ncols = k + 1;
                sm.rows = total;
            }
            __syncthreads();
        } else {
            // Cartesian product with a relation of 1 or 2 columns: M_p,
            // its diagonal, or the row of a constant
            const int32_t *rel0;
            const int32_t *rel1 = nullptr;
            int64_t m;
            int rc;
            if (S.kind == GSMAT_STEP_EXPAND_S || S.kind == GSMAT_STEP_EXPAND_O) {
                const int side = S.kind == GSMAT_STEP_EXPAND_S ? 0 : 1;
                rel0 = a.sv.side[side].val + S.c_first;
                m = S.c_last - S.c_first;
                rc = 1;
            } else if (S.diag) {
                int32_t *dg = cta_alloc(a, sm, sizeof(int32_t) * (size_t)(p0.nnz > 0 ? p0.nnz : 1));
                if (!dg) {
                    if (tid == 0) sm.status = BR_OVERFLOW;
                    __syncthreads();
                    break;
                }
                const int32_t *kk = a.sv.side[0].key + p0.ent_base;
                const int32_t *vv = a.sv.side[0].val + p0.ent_base;
                int64_t carry = 0;
                for (int64_t base = 0; base < p0.nnz; base += BLOCK) {
                    const int64_t i = base + tid;
                    const bool f = i < p0.nnz && kk[i] == vv[i];
                    int64_t tot;
                    const int64_t ex = cta_scan(sm, f ? 1 : 0, &tot);
                    if (f) dg[carry + ex] = kk[i];
                    carry += tot;
                }
                rel0 = dg;
                m = carry;
                rc = 1;
            } else {
                const PredSide &pp = S.swap ? p1 : p0;
                rel0 = a.sv.side[S.swap].key + pp.ent_base;
                rel1 = a.sv.side[S.swap].val + pp.ent_base;
                m = pp.nnz;
                rc = 2;
            }
            if (unit) {
                __syncthreads();
                if (tid == 0) {
                    sm.col[0] = rel0;
                    if (rc == 2) sm.col[1] = rel1;
                    sm.ncols = rc;
                    sm.rows = m;
                }
                __syncthreads();
                continue;
            }
            const int64_t total = n * m;
            if (total > a.max_rows) {
                if (tid == 0) sm.status = BR_OVERFLOW;
                __syncthreads();
                break;
            }
            int32_t *out = total > 0 ? cta_alloc(a, sm, sizeof(int32_t) * (size_t)total * (k + rc)) : nullptr;
            if (total > 0 && !out) {
                if (tid == 0) sm.status = BR_OVERFLOW;
                __syncthreads();
                break;
            }
            for (int64_t j = tid; j < total; j += BLOCK) {
                const int64_t r = j / m, qq = j - r * m;
                for (int c = 0; c < k; ++c) out[(size_t)c * total + j] = sm.col[c][r];
                out[(size_t)k * total + j] = rel0[qq];
                if (rc == 2) out[(size_t)(k + 1) * total + j] = rel1[qq];
            }
            __syncthreads();
            if (tid == 0) {
                for (int c = 0; c < k + rc; ++c) sm.col[c] = out + (size_t)c * total;
                sm.ncols = k + rc;
                sm.rows = total;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    // result: columns in variable order, rows ascending
    BResult &R = a.results[q];
    const int64_t rows = sm.rows;
    const int V = Q.n_vars;
    if (sm.status != BR_OK) {
        if (tid == 0) {
            R.status = sm.status;
            R.rows = 0;
            R.ncols = V;
        }
        return;
    }
    if (rows == 0 || sm.ncols != V || Q.m_sort == 0 || rows <= 1) {
        if (tid == 0) {
            R.status = BR_OK;
            R.rows = (sm.ncols == V) ? rows : 0;
            R.ncols = V;
            for (int v = 0; v < V; ++v) R.col[v] = (sm.ncols == V) ? sm.col[Q.col_of_var[v]] : nullptr;
        }
        return;
    }
    const int m = Q.m_sort;
    if (rows > kSmemSortRows || m * a.bits > 64) {
        if (tid == 0) {
            R.status = BR_NEEDS_SORT;  // finished by the multi-CTA reorder
            R.rows = rows;
            R.ncols = V;
            for (int v = 0; v < V; ++v) R.col[v] = sm.col[Q.col_of_var[v]];
        }
        return;
    }
    // shared-memory sort of (key over variables 0..m-1, row) pairs; the row
    // index breaks ties, so the order is the stable one
    int n2 = 1;
    while (n2 < rows) n2 <<= 1;
    for (int i = tid; i < n2; i += BLOCK) {
        unsigned long long key = ~0ull;
        if (i < rows) {
            key = 0;
            for (int v = 0; v < m; ++v) key = (key << a.bits) | (uint32_t)sm.col[Q.col_of_var[v]][i];
        }
        sm.skey[i] = key;
        sm.sidx[i] = (uint16_t)(i < rows ? i : 0xffff);
    }
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < n2; i += BLOCK) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long ki = sm.skey[i], kj = sm.skey[j];
                    const uint16_t ii = sm.sidx[i], ij = sm.sidx[j];
                    const bool gt = ki > kj || (ki == kj && ii > ij);
                    if (gt == up) {
                        sm.skey[i] = kj;
                        sm.skey[j] = ki;
                        sm.sidx[i] = ij;
                        sm.sidx[j] = ii;
                    }
                }
            }
            __syncthreads();
        }
    }
    int32_t *out = cta_alloc(a, sm, sizeof(int32_t) * (size_t)rows * V);
    if (!out) {
        if (tid == 0) {
            R.status = BR_OVERFLOW;
            R.rows = 0;
            R.ncols = V;
        }
        return;
    }
    for (int64_t i = tid; i < rows; i += BLOCK) {
        const int r = sm.sidx[i];
        for (int v = 0; v < V; ++v) out[(size_t)v * rows + i] = sm.col[Q.col_of_var[v]][r];
    }
    __syncthreads();
    if (tid == 0) {
        R.status = BR_OK;
        R.rows = rows;
        R.ncols = V;
        for (int v = 0; v < V; ++v) R.col[v] = out + (size_t)v * rows;
    }
}

template <int BLOCK, int EPT>
__global__ void __launch_bounds__(BLOCK) batch_kernel(BatchArgs a) {
    __shared__ CtaShared<BLOCK> sm;
    while (true) {
        if (threadIdx.x == 0) sm.q = (int)atomicAdd(a.queue_head, 1u);
        __syncthreads();
        const int q = sm.q;
        __syncthreads();
        if (q >= a.n_queries) break;
        run_query<BLOCK, EPT>(a, sm, q);
        __syncthreads();
    }
}

// Segmented reorder of many result tables at once (the batch's large
// results): key = segment id above the segment's leading variables, payload
// = row of the concatenation.

// keys[g] = variables [vb, ve) of source row src = perm_in[g] (or g),
// packed most significant first, with the source's segment index above
// them when seg_shift >= 0; perm_out[g] = g when perm_in is null.
// Segment of row g: the last s with start[s] <= g (start = the segments'
// first rows, ascending; a compact array, cached, unlike the descriptors).
__device__ __forceinline__ int seg_of(const int64_t *__restrict__ start, int n_segs, int64_t g) {
    int lo = 0, hi = n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// idx_bits > 0: the source position rides in the key's low idx_bits bits
// (key << idx_bits | src) and perm_out is not written.
__global__ void seg_pack_kernel(const SegDesc *__restrict__ segs, int n_segs, int bits, int vb, int ve, int seg_shift,
                                int idx_bits, const uint32_t *__restrict__ perm_in, int64_t total,
                                uint64_t *__restrict__ keys, uint32_t *__restrict__ perm_out) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t src = perm_in ? (int64_t)__ldg(perm_in + g) : g;
        const int lo = seg_of(reinterpret_cast<const int64_t *>(segs + n_segs), n_segs, src);
        const SegDesc &s = segs[lo];
        const int64_t r = src - s.row_off;
        uint64_t key = 0;
        for (int v = vb; v < ve; ++v) key = (key << bits) | (uint32_t)__ldg(s.col[v] + r);
        if (seg_shift >= 0) key |= (uint64_t)lo << seg_shift;
        if (idx_bits > 0) {
            keys[g] = (key << idx_bits) | (uint64_t)src;
        } else {
            keys[g] = key;
            if (!perm_in) perm_out[g] = (uint32_t)g;
        }
    }
}

// Carried columns: keys[g] = (segment << kb) | the key variables [0, m) of
// row g (`bits` each), pay[g] = the segment's other variables [m, V) packed
// the same way (rows in segment order, before the sort).
__global__ void seg_pack_wide_kernel(const SegDesc *__restrict__ segs, int n_segs, int bits, int m, int kb,
                                     int64_t total, uint64_t *__restrict__ keys, uint64_t *__restrict__ pay) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int lo = seg_of(reinterpret_cast<const int64_t *>(segs + n_segs), n_segs, g);
        const SegDesc &s = segs[lo];
        const int64_t r = g - s.row_off;
        uint64_t key = 0, p = 0;
        for (int v = 0; v < m; ++v) key = (key << bits) | (uint32_t)__ldg(s.col[v] + r);
        for (int v = m; v < s.V; ++v) p = (p << bits) | (uint32_t)__ldg(s.col[v] + r);
        keys[g] = ((uint64_t)lo << kb) | key;
        pay[g] = p;
    }
}

// The sorted rows of every segment from the carried key and payload (the
// segment index is the key's most significant field, so each segment keeps
// its positions).
__global__ void seg_unpack_wide_kernel(const SegDesc *__restrict__ segs, int n_segs, int bits, int m, int64_t total,
                                       const uint64_t *__restrict__ keys, const uint64_t *__restrict__ pay) {
    const uint64_t fmask = (1ull << bits) - 1;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int lo = seg_of(reinterpret_cast<const int64_t *>(segs + n_segs), n_segs, g);
        const SegDesc &s = segs[lo];
        const int64_t i = g - s.row_off;
        const uint64_t key = __ldg(keys + g), p = __ldg(pay + g);
        for (int v = 0; v < m; ++v) s.out[(size_t)v * s.rows + i] = (int32_t)((key >> ((m - 1 - v) * bits)) & fmask);
        const int nr = s.V - m;
        for (int v = m; v < s.V; ++v) {
            s.out[(size_t)v * s.rows + i] = (int32_t)((p >> ((nr - 1 - (v - m)) * bits)) & fmask);
        }
    }
}

__global__ void key_low_bits_kernel(const uint64_t *__restrict__ keys, int idx_bits, int64_t total,
                                    uint32_t *__restrict__ perm) {
    const uint64_t mask = (1ull << idx_bits) - 1;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        perm[g] = (uint32_t)(__ldg(keys + g) & mask);
    }
}

__global__ void seg_gather_kernel(const SegDesc *__restrict__ segs, int n_segs, int64_t total,
                                  const uint32_t *__restrict__ perm) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
        const int lo = seg_of(reinterpret_cast<const int64_t *>(segs + n_segs), n_segs, p);
        const SegDesc &s = segs[lo];
        const int64_t r = (perm ? (int64_t)__ldg(perm + p) : p) - s.row_off;  // source row (same segment)
        const int64_t i = p - s.row_off;                          // destination row
        for (int v = 0; v < s.V; ++v) s.out[(size_t)v * s.rows + i] = __ldg(s.col[v] + r);
    }
}

}  // namespace

int launch_seg_pack(const SegDesc *segs, int n_segs, int bits, int vb, int ve, int seg_shift, int idx_bits,
                    const uint32_t *perm_in, int64_t total, uint64_t *keys, uint32_t *perm_out, cudaStream_t st) {
    if (total <= 0) return GSMAT_OK;
    KernelTimer t("seg_pack", st, (double)total * (12.0 + 4.0 * (ve - vb)), (double)total);
    seg_pack_kernel<<<grid_1d(total, 256), 256, 0, st>>>(segs, n_segs, bits, vb, ve, seg_shift, idx_bits, perm_in,
                                                         total, keys, perm_out);
    GS_LAUNCH_CHECK();
    t.stop();
    return GSMAT_OK;
}

int launch_seg_pack_wide(const SegDesc *segs, int n_segs, int bits, int m, int kb, int64_t total, uint64_t *keys,
                         uint64_t *pay, cudaStream_t st) {
    if (total <= 0) return GSMAT_OK;
    seg_pack_wide_kernel<<<grid_1d(total, 256), 256, 0, st>>>(segs, n_segs, bits, m, kb, total, keys, pay);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

int launch_seg_unpack_wide(const SegDesc *segs, int n_segs, int bits, int m, int64_t total, const uint64_t *keys,
                           const uint64_t *pay, cudaStream_t st) {
    if (total <= 0) return GSMAT_OK;
    seg_unpack_wide_kernel<<<grid_1d(total, 256), 256, 0, st>>>(segs, n_segs, bits, m, total, keys, pay);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

int launch_key_low_bits(const uint64_t *keys, int idx_bits, int64_t total, uint32_t *perm, cudaStream_t st) {
    if (total <= 0) return GSMAT_OK;
    key_low_bits_kernel<<<grid_1d(total, 256), 256, 0, st>>>(keys, idx_bits, total, perm);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

int launch_seg_gather(const SegDesc *segs, int n_segs, int64_t total, const uint32_t *perm, cudaStream_t st) {
    if (total <= 0) return GSMAT_OK;
    KernelTimer t("seg_gather", st, (double)total * 36.0, (double)total);
    seg_gather_kernel<<<grid_1d(total, 256), 256, 0, st>>>(segs, n_segs, total, perm);
    GS_LAUNCH_CHECK();
    t.stop();
    return GSMAT_OK;
}

int launch_batch_kernel(const BatchArgs &a, int block, int expand_slots, int grid, cudaStream_t st) {
    const bool four = expand_slots == 4;
    if (block == 128) {
        if (four) batch_kernel<128, 4><<<grid, 128, 0, st>>>(a);
        else batch_kernel<128, 1><<<grid, 128, 0, st>>>(a);
    } else if (block == 512) {
        if (four) batch_kernel<512, 4><<<grid, 512, 0, st>>>(a);
        else batch_kernel<512, 1><<<grid, 512, 0, st>>>(a);
    } else {
        if (four) batch_kernel<256, 4><<<grid, 256, 0, st>>>(a);
        else batch_kernel<256, 1><<<grid, 256, 0, st>>>(a);
    }
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

}  // namespace gs
