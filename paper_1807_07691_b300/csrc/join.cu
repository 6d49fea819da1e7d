// Kernels of one SM-based join step (Alg. 3, Sec. 6.3) on the GPU.
//
// The paper's GPU join (Sec. 7.2) assigns one thread to each non-zero row of
// the left matrix and pre-computes per-row output counts N and offsets P
// (Alg. 4).  Here the count and the offset scan are fused into one
// single-pass kernel, and the expansion is output-slot parallel: each CTA
// owns a fixed slab of output rows and finds the parent row of each slot by
// a search over the offsets, so a hub row with 10^6 matches is spread over
// many CTAs instead of serialising one thread (power-law degrees, Sec. 1).
// Rows whose other join variables must also match (Alg. 3, the "other join
// variables" test) are kept by a membership filter with single-pass
// prefix-sum compaction, which preserves row order.
#include <atomic>

#include "join.cuh"
#include "select.cuh"

namespace gs {
namespace {

// ---------------------------------------------------------------------------
// count + scan

constexpr int kCsBlock = 256;
constexpr int kCsItems = 8;
constexpr int kCsTile = kCsBlock * kCsItems;

// Items are warp-striped (item j of lane l of warp w is row
// tile * kCsTile + w * 32 * kCsItems + 32 j + l), so loads and stores are
// coalesced; the tile's prefix runs in that order: a warp scan per j, the
// warp's running total across j, then the warps' totals.
__global__ void __launch_bounds__(kCsBlock) count_scan_kernel(SideView sv, PredSide ps,
                                                              const int32_t *__restrict__ x, int64_t n,
                                                              int64_t *__restrict__ off, int32_t *__restrict__ first,
                                                              int64_t *__restrict__ d_total, LookbackScratch ls) {
    __shared__ int tile_sm;
    __shared__ int64_t scan_sm[kCsBlock / 32 + 1];
    __shared__ int64_t prefix_sm;
    const int tile = acquire_tile_id(ls, &tile_sm);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i0 = (int64_t)tile * kCsTile + (int64_t)warp * (32 * kCsItems) + lane;
    int32_t xv[kCsItems];
    bool ok[kCsItems];
#pragma unroll
    for (int j = 0; j < kCsItems; ++j) {
        ok[j] = i0 + 32 * j < n;
        xv[j] = ok[j] ? __ldg(x + i0 + 32 * j) : 0;
    }
    int2 rr[kCsItems];
    row_ranges<kCsItems>(sv, ps, xv, ok, rr);
    // exclusive prefix of every item inside its warp's part of the tile
    int64_t ex[kCsItems];
    int64_t wrun = 0;
#pragma unroll
    for (int j = 0; j < kCsItems; ++j) {
        const int64_t c = rr[j].y - rr[j].x;
        const int64_t inc = warp_inclusive_sum(c);
        ex[j] = wrun + inc - c;
        wrun += __shfl_sync(0xffffffffu, inc, 31);
    }
    int64_t tot;
    const int64_t wex = block_exclusive_sum<kCsBlock>(lane == 0 ? wrun : 0, scan_sm, &tot);
    const int64_t wbase = __shfl_sync(0xffffffffu, wex, 0);
    const int64_t pre = tile_lookback(ls, tile, tot, &prefix_sm);
#pragma unroll
    for (int j = 0; j < kCsItems; ++j) {
        if (ok[j]) {
            off[i0 + 32 * j] = pre + wbase + ex[j];
            first[i0 + 32 * j] = rr[j].x;
        }
    }
    if (tile == (int)gridDim.x - 1 && threadIdx.x == 0) {
        off[n] = pre + tot;
        *d_total = pre + tot;
    }
}

// ---------------------------------------------------------------------------
// expand
//
// Load balance: the merge of the row-end sequence off[1..n] with the output
// slots 0..total-1 is cut into pieces of kExItems items (rows + slots), so a
// CTA never sees more than kExItems parent rows, however many input rows
// have no match.  A partition kernel finds every cut by a merge-path search;
// the expand kernel stages its piece of the offsets in shared memory and
// finds each slot's parent by a shared-memory binary search.

constexpr int kExBlock = 256;

// Number of rows whose end off[r + 1] precedes output slot diag - a in the
// merge, for the first `diag` merged items (rows win ties).
__device__ __forceinline__ int64_t merge_path(const int64_t *__restrict__ off, int64_t n_rows, int64_t total,
                                              int64_t diag) {
    int64_t lo = diag - total > 0 ? diag - total : 0;
    int64_t hi = diag < n_rows ? diag : n_rows;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid + 1) <= diag - 1 - mid) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void expand_partition_kernel(const int64_t *__restrict__ off, int64_t n_rows, int64_t total, int64_t n_parts,
                                        int items, int64_t *__restrict__ cuts) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p > n_parts) return;
    int64_t diag = p * items;
    if (diag > n_rows + total) diag = n_rows + total;
    cuts[p] = merge_path(off, n_rows, total, diag);
}

struct ExpandArgs {
    int items;           // rows + slots per CTA (dynamic shared memory sized for it)
    const int32_t *val;  // the side's entry array
    Cols in;
    int k;
    int64_t n_in;
    const int64_t *off;
    const int32_t *first;
    int64_t total;
    const int64_t *cuts;
    OutCols out;
};

// Each thread writes groups of 4 consecutive output slots aligned to 4:
// one binary search finds the group's first parent, the next slots step
// forward through the offsets, and a group wholly inside the CTA's slab is
// written with one 16-byte store per column (columns are 256-byte aligned).
__global__ void __launch_bounds__(kExBlock) expand_kernel(ExpandArgs a) {
    extern __shared__ __align__(16) unsigned char ex_smem[];
    int64_t *soff = reinterpret_cast<int64_t *>(ex_smem);            // items + 2
    int32_t *sfirst = reinterpret_cast<int32_t *>(soff + a.items + 2);  // items + 1
    const int64_t d0 = (int64_t)blockIdx.x * a.items;
    const int64_t d1 = d0 + a.items < a.n_in + a.total ? d0 + a.items : a.n_in + a.total;
    const int64_t r0 = __ldg(a.cuts + blockIdx.x);
    const int64_t r1 = __ldg(a.cuts + blockIdx.x + 1);
    const int64_t j0 = d0 - r0, j1 = d1 - r1;  // output slots [j0, j1)
    if (j1 <= j0) return;
    // parents of the slots lie in [r0, r_last]
    const int64_t r_last = r1 < a.n_in ? r1 : a.n_in - 1;
    const int nr = (int)(r_last - r0 + 1);
    for (int i = threadIdx.x; i <= nr; i += kExBlock) soff[i] = __ldg(a.off + r0 + i);
    for (int i = threadIdx.x; i < nr; i += kExBlock) sfirst[i] = __ldg(a.first + r0 + i);
    __syncthreads();
    const int k = a.k;
    const int32_t *__restrict__ val = a.val;
    const int64_t g0 = j0 >> 2, g1 = (j1 + 3) >> 2;
    for (int64_t g = g0 + threadIdx.x; g < g1; g += kExBlock) {
        const int64_t jb = g << 2;
        const int64_t js = jb > j0 ? jb : j0;  // first slot of the group in the slab
        // parent of js: largest i in [0, nr) with soff[i] <= js
        int lo = 0, hi = nr - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (soff[mid] <= js) lo = mid; else hi = mid - 1;
        }
        int par[4];
        int32_t nb[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t j = jb + t;
            par[t] = lo;
            nb[t] = 0;
            if (j >= js && j < j1) {
                while (lo + 1 < nr && soff[lo + 1] <= j) ++lo;
                par[t] = lo;
                nb[t] = __ldg(val + sfirst[lo] + (j - soff[lo]));
            }
        }
        if (jb >= j0 && jb + 4 <= j1) {
            for (int c = 0; c < k; ++c) {
                const int32_t *col = a.in.c[c] + r0;
                reinterpret_cast<int4 *>(a.out.c[c])[g] =
                    make_int4(__ldg(col + par[0]), __ldg(col + par[1]), __ldg(col + par[2]), __ldg(col + par[3]));
            }
            reinterpret_cast<int4 *>(a.out.c[k])[g] = make_int4(nb[0], nb[1], nb[2], nb[3]);
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int64_t j = jb + t;
                if (j < js || j >= j1) continue;
                for (int c = 0; c < k; ++c) a.out.c[c][j] = __ldg(a.in.c[c] + r0 + par[t]);
                a.out.c[k][j] = nb[t];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// product of independent expansions

constexpr int kPcBlock = 256;
constexpr int kPcItems = 4;
constexpr int kPcTile = kPcBlock * kPcItems;
constexpr uint64_t kProdSaturate = uint64_t(1) << 32;  // already past the row limit of a table

__device__ __forceinline__ uint64_t sat_mul(uint64_t c, uint64_t l) {
    return (l != 0 && c > kProdSaturate / l) ? kProdSaturate : c * l;
}

// Count + scan, laid out like count_scan_kernel (warp-striped items, warp
// scans, the CTA's warp totals, decoupled look-back across tiles).
__global__ void __launch_bounds__(kPcBlock) product_count_scan_kernel(StoreView sv, ProdSpec spec, Cols in, int64_t n,
                                                                      int64_t *__restrict__ off,
                                                                      int32_t *__restrict__ first,
                                                                      int32_t *__restrict__ len,
                                                                      int64_t *__restrict__ d_total, LookbackScratch ls) {
    __shared__ int tile_sm;
    __shared__ int64_t scan_sm[kPcBlock / 32 + 1];
    __shared__ int64_t prefix_sm;
    const int tile = acquire_tile_id(ls, &tile_sm);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i0 = (int64_t)tile * kPcTile + (int64_t)warp * (32 * kPcItems) + lane;
    uint64_t cnt[kPcItems];
    bool ok[kPcItems];
#pragma unroll
    for (int j = 0; j < kPcItems; ++j) {
        ok[j] = i0 + 32 * j < n;
        cnt[j] = ok[j] ? 1 : 0;
    }
    for (int fi = 0; fi < spec.nf; ++fi) {
        const ProdFactor &f = spec.f[fi];
        if (f.kind != kProdRow) {
#pragma unroll
            for (int j = 0; j < kPcItems; ++j) cnt[j] = sat_mul(cnt[j], f.len);
            continue;
        }
        int32_t xv[kPcItems];
#pragma unroll
        for (int j = 0; j < kPcItems; ++j) xv[j] = ok[j] ? __ldg(in.c[f.xcol] + i0 + 32 * j) : 0;
        int2 rr[kPcItems];
        row_ranges<kPcItems>(sv.side[f.side], f.ps, xv, ok, rr);
#pragma unroll
        for (int j = 0; j < kPcItems; ++j) {
            const uint64_t l = (uint64_t)(rr[j].y - rr[j].x);
            cnt[j] = sat_mul(cnt[j], l);
            if (ok[j]) {
                first[(int64_t)f.slot * n + i0 + 32 * j] = rr[j].x;
                len[(int64_t)f.slot * n + i0 + 32 * j] = rr[j].y - rr[j].x;
            }
        }
    }
    int64_t ex[kPcItems];
    int64_t wrun = 0;
#pragma unroll
    for (int j = 0; j < kPcItems; ++j) {
        const int64_t c = (int64_t)cnt[j];
        const int64_t inc = warp_inclusive_sum(c);
        ex[j] = wrun + inc - c;
        wrun += __shfl_sync(0xffffffffu, inc, 31);
    }
    int64_t tot;
    const int64_t wex = block_exclusive_sum<kPcBlock>(lane == 0 ? wrun : 0, scan_sm, &tot);
    const int64_t wbase = __shfl_sync(0xffffffffu, wex, 0);
    const int64_t pre = tile_lookback(ls, tile, tot, &prefix_sm);
#pragma unroll
    for (int j = 0; j < kPcItems; ++j) {
        if (ok[j]) off[i0 + 32 * j] = pre + wbase + ex[j];
    }
    if (tile == (int)gridDim.x - 1 && threadIdx.x == 0) {
        off[n] = pre + tot;
        *d_total = pre + tot;
    }
}

struct ProductArgs {
    int items;  // rows + slots per CTA (dynamic shared memory sized for it)
    StoreView sv;
    ProdSpec spec;
    Cols in;
    int k;
    int64_t n_in;
    const int64_t *off;
    const int32_t *first;
    const int32_t *len;
    int64_t total;
    const int64_t *cuts;
    OutCols out;
};

// Slots are partitioned as in expand_kernel (merge path of row ends and
// slots, kExItems per CTA, the CTA's offsets staged in shared memory) and
// taken in groups of 4 aligned slots as there: one search per group, 16-byte
// stores for a group wholly inside the slab.
__device__ __forceinline__ int32_t product_value(const ProductArgs &a, const ProdFactor &f, int64_t r, uint32_t &q,
                                                 int32_t *second) {
    if (f.kind == kProdRow) {
        const int64_t at = (int64_t)f.slot * a.n_in + r;
        const uint32_t l = (uint32_t)__ldg(a.len + at);
        const uint32_t qq = q / l;
        const uint32_t idx = q - qq * l;
        q = qq;
        return __ldg(a.sv.side[f.side].val + __ldg(a.first + at) + idx);
    }
    const uint32_t qq = fastdiv_quot(q, f.div);
    const uint32_t idx = q - qq * f.len;
    q = qq;
    if (f.kind == kProdPairs) *second = __ldg(f.b + idx);
    return __ldg(f.a + idx);
}

__global__ void __launch_bounds__(kExBlock) product_kernel(ProductArgs a) {
    extern __shared__ __align__(16) unsigned char pr_smem[];
    int64_t *soff = reinterpret_cast<int64_t *>(pr_smem);  // items + 2
    const int64_t d0 = (int64_t)blockIdx.x * a.items;
    const int64_t d1 = d0 + a.items < a.n_in + a.total ? d0 + a.items : a.n_in + a.total;
    const int64_t r0 = __ldg(a.cuts + blockIdx.x);
    const int64_t r1 = __ldg(a.cuts + blockIdx.x + 1);
    const int64_t j0 = d0 - r0, j1 = d1 - r1;
    if (j1 <= j0) return;
    const int64_t r_last = r1 < a.n_in ? r1 : a.n_in - 1;
    const int nr = (int)(r_last - r0 + 1);
    for (int i = threadIdx.x; i <= nr; i += kExBlock) soff[i] = __ldg(a.off + r0 + i);
    __syncthreads();
    const int nf = a.spec.nf;
    const int64_t g0 = j0 >> 2, g1 = (j1 + 3) >> 2;
    for (int64_t g = g0 + threadIdx.x; g < g1; g += kExBlock) {
        const int64_t jb = g << 2;
        const int64_t js = jb > j0 ? jb : j0;
        int lo = 0, hi = nr - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (soff[mid] <= js) lo = mid; else hi = mid - 1;
        }
        int par[4];
        uint32_t q0[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t j = jb + t;
            if (j >= js && j < j1) {
                while (lo + 1 < nr && soff[lo + 1] <= j) ++lo;
            }
            par[t] = lo;
            q0[t] = (uint32_t)(j - soff[lo]);  // < N_r <= total < 2^32 for the slab's slots
        }
        const bool full = jb >= j0 && jb + 4 <= j1;
        if (full) {
            for (int c = 0; c < a.k; ++c) {
                const int32_t *col = a.in.c[c] + r0;
                reinterpret_cast<int4 *>(a.out.c[c])[g] =
                    make_int4(__ldg(col + par[0]), __ldg(col + par[1]), __ldg(col + par[2]), __ldg(col + par[3]));
            }
            uint32_t q[4] = {q0[0], q0[1], q0[2], q0[3]};
            for (int fi = nf - 1; fi >= 0; --fi) {
                const ProdFactor &f = a.spec.f[fi];
                int32_t v[4], w[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) v[t] = product_value(a, f, r0 + par[t], q[t], &w[t]);
                reinterpret_cast<int4 *>(a.out.c[f.out0])[g] = make_int4(v[0], v[1], v[2], v[3]);
                if (f.kind == kProdPairs) reinterpret_cast<int4 *>(a.out.c[f.out0 + 1])[g] = make_int4(w[0], w[1], w[2], w[3]);
            }
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int64_t j = jb + t;
                if (j < js || j >= j1) continue;
                const int64_t r = r0 + par[t];
                for (int c = 0; c < a.k; ++c) a.out.c[c][j] = __ldg(a.in.c[c] + r);
                uint32_t q = q0[t];
                for (int fi = nf - 1; fi >= 0; --fi) {
                    const ProdFactor &f = a.spec.f[fi];
                    int32_t w = 0;
                    a.out.c[f.out0][j] = product_value(a, f, r, q, &w);
                    if (f.kind == kProdPairs) a.out.c[f.out0 + 1][j] = w;
                }
            }
        }
    }
}

// Row j of a product of fixed lists takes entry (j / inner_i) mod len_i of
// factor i (inner_i = product of the lengths of the factors nested inside
// it).  A thread writes 4 consecutive rows of every column with one 16-byte
// store each (columns are 256-byte aligned); the last total mod 4 rows are
// written one by one.
__global__ void __launch_bounds__(256) product_fixed_kernel(ProdSpec spec, uint32_t total, OutCols out) {
    const int nf = spec.nf;
    const int64_t n4 = (int64_t)(total >> 2);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n4; g += stride) {
        const uint32_t j0 = (uint32_t)(g << 2);
        for (int fi = 0; fi < nf; ++fi) {
            const ProdFactor &f = spec.f[fi];
            int4 va, vb;
            int32_t *pa = &va.x, *pb = &vb.x;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint32_t q = fastdiv_quot(j0 + t, f.inner);
                const uint32_t idx = q - fastdiv_quot(q, f.div) * f.len;
                pa[t] = __ldg(f.a + idx);
                if (f.kind == kProdPairs) pb[t] = __ldg(f.b + idx);
            }
            reinterpret_cast<int4 *>(out.c[f.out0])[g] = va;
            if (f.kind == kProdPairs) reinterpret_cast<int4 *>(out.c[f.out0 + 1])[g] = vb;
        }
    }
    const uint32_t rest = total & 3u;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < (int64_t)rest) {
        const uint32_t j = (uint32_t)(n4 << 2) + (uint32_t)t;
        for (int fi = 0; fi < nf; ++fi) {
            const ProdFactor &f = spec.f[fi];
            const uint32_t q = fastdiv_quot(j, f.inner);
            const uint32_t idx = q - fastdiv_quot(q, f.div) * f.len;
            out.c[f.out0][j] = __ldg(f.a + idx);
            if (f.kind == kProdPairs) out.c[f.out0 + 1][j] = __ldg(f.b + idx);
        }
    }
}

// ---------------------------------------------------------------------------
// filter (membership test of (s, o) in the predicate) + compaction

struct FilterOp {
    int short_row;  // rows this short are searched directly, without looking up the other side
    SideView s0, s1;
    PredSide ps_s, ps_o;
    ValueSrc s, o;
    Cols in;
    int k;
    OutCols out;
    __device__ bool flag(int64_t i) const {
        const int32_t x = s.at(i), y = o.at(i);
        const int2 a = row_range(s0, ps_s, x);
        const int la = a.y - a.x;
        if (la <= 0) return false;
        if (la <= short_row) return sorted_contains(s0.val, a.x, a.y, y);
        const int2 b = row_range(s1, ps_o, y);
        const int lb = b.y - b.x;
        if (lb <= 0) return false;
        if (la <= lb) return sorted_contains(s0.val, a.x, a.y, y);
        return sorted_contains(s1.val, b.x, b.y, x);
    }
    __device__ void emit(int64_t i, int64_t j) const {
        for (int c = 0; c < k; ++c) out.c[c][j] = __ldg(in.c[c] + i);
    }
};

// ---------------------------------------------------------------------------
// intersect-expand: a new variable bound by two patterns at once.  Row i's
// candidates are the intersection of two sorted entry lists (the row of
// a_i in one predicate side and the row of b_i in another); one warp per
// input row walks the shorter list in chunks of 32, each lane binary
// searches its element in the part of the longer list not yet passed,
// and ballot / popc give every match its output position.  Matches come
// out ascending, the order an expand followed by a filter produces.

struct IsectSrc {
    SideView sa, sb;
    PredSide pa, pb;
    ValueSrc a, b;
};

// Count (out == nullptr) or write the intersection of row i; returns the
// count (in every lane).  k parent columns are copied for each match.
__device__ __forceinline__ int warp_intersect_row(const IsectSrc &s, int64_t i, int64_t out_base, const Cols &in,
                                                  int k, OutCols *out) {
    if (!out) return warp_intersect(s.sa, s.pa, s.a.at(i), s.sb, s.pb, s.b.at(i), [](int, int32_t) {});
    return warp_intersect(s.sa, s.pa, s.a.at(i), s.sb, s.pb, s.b.at(i), [&](int r, int32_t v) {
        const int64_t j = out_base + r;
        for (int c = 0; c < k; ++c) out->c[c][j] = __ldg(in.c[c] + i);
        out->c[k][j] = v;
    });
}

__global__ void __launch_bounds__(256) isect_count_kernel(IsectSrc s, int64_t n, int32_t *__restrict__ counts) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        Cols none;
        const int c = warp_intersect_row(s, i, 0, none, 0, nullptr);
        if ((threadIdx.x & 31) == 0) counts[i] = c;
    }
}

__global__ void __launch_bounds__(256) isect_write_kernel(IsectSrc s, int64_t n, const int64_t *__restrict__ off,
                                                          Cols in, int k, OutCols out) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        if (__ldg(off + i + 1) == __ldg(off + i)) continue;  // warp-uniform
        warp_intersect_row(s, i, __ldg(off + i), in, k, &out);
    }
}

// ---------------------------------------------------------------------------
// Cartesian product

__global__ void __launch_bounds__(256) cross_kernel(Cols in, int k, Cols rel, int rc, uint32_t m, uint64_t total,
                                                    OutCols out) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < total; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t jj = (uint32_t)j;
        const uint32_t r = jj / m;
        const uint32_t q = jj - r * m;
        for (int c = 0; c < k; ++c) out.c[c][jj] = __ldg(in.c[c] + r);
        for (int c = 0; c < rc; ++c) out.c[k + c][jj] = __ldg(rel.c[c] + q);
    }
}

struct DiagOp {
    const int32_t *key, *val;
    int32_t *out;
    __device__ bool flag(int64_t i) const { return key[i] == val[i]; }
    __device__ void emit(int64_t i, int64_t j) const { out[j] = key[i]; }
};

__global__ void const_lookup_kernel(StoreView sv, const PredSide *__restrict__ sides, int n_pred,
                                    const int32_t *__restrict__ req, int n_req, int32_t *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_req) return;
    const int slot = req[3 * i], side = req[3 * i + 1], x = req[3 * i + 2];
    int2 r = make_int2(0, 0);
    if (slot >= 0 && slot < n_pred && (side == 0 || side == 1)) {
        r = row_range(side == 0 ? sv.side[0] : sv.side[1], sides[side * n_pred + slot], x);
    }
    out[2 * i] = r.x;
    out[2 * i + 1] = r.y;
}

// ---------------------------------------------------------------------------
// row gathers and layout conversion

__global__ void interleave_kernel(Cols in, int k, int64_t n, int32_t *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < k; ++c) dst[i * k + c] = __ldg(in.c[c] + i);
    }
}

__global__ void copy_cols_kernel(Cols in, int k, int64_t n, OutCols out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < k; ++c) out.c[c][i] = __ldg(in.c[c] + i);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers

int launch_count_scan(const StoreView &sv, int side, const PredSide &ps, const int32_t *x, int64_t n, int64_t *off,
                      int32_t *first, int64_t *d_total, int *err, cudaStream_t st) {
    if (n <= 0) {
        GS_CUDA(cudaMemsetAsync(off, 0, sizeof(int64_t), st));
        GS_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int64_t), st));
        return GSMAT_OK;
    }
    const int64_t ntiles = (n + kCsTile - 1) / kCsTile;
    if (ntiles > INT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "count over %lld rows", (long long)n);
    LookbackBuf lb;
    GS_TRY(lb.make(ntiles, st, err));
    // algorithmic bytes: bound column, one row lookup (8 B), offsets + first
    KernelTimer t("count_scan", st, (double)n * (4.0 + 8.0 + 8.0 + 4.0), (double)n);
    count_scan_kernel<<<(unsigned)ntiles, kCsBlock, 0, st>>>(sv.side[side], ps, x, n, off, first, d_total, lb.view);
    GS_LAUNCH_CHECK();
    t.stop();
    return GSMAT_OK;
}

// Dynamic shared memory of the expand / product kernels for `items` per CTA
// (above the default 48 KB the limit is raised once per device).
template <class Kernel>
int prepare_items_smem(Kernel kernel, int items, size_t bytes, std::atomic<int> *done_bytes) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (bytes > 48 * 1024 && done_bytes[dev].load(std::memory_order_acquire) < (int)bytes) {
        GS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        done_bytes[dev].store((int)bytes, std::memory_order_release);
    }
    (void)items;
    return GSMAT_OK;
}

int tile_config_check(const TileConfig &tc) {
    const int e = tc.expand_items;
    if (e != 512 && e != 1024 && e != 2048 && e != 4096 && e != 8192) {
        return set_error(GSMAT_ERR_INVALID_ARG, "expand_items %d (512, 1024, 2048, 4096 or 8192)", e);
    }
    if (tc.short_row < 1 || tc.short_row > 4096) {
        return set_error(GSMAT_ERR_INVALID_ARG, "short_row %d outside [1, 4096]", tc.short_row);
    }
    return GSMAT_OK;
}

int launch_expand(const StoreView &sv, int side, const Cols &in, int k, int64_t n_in, const int64_t *off,
                  const int32_t *first, int64_t total, OutCols out, cudaStream_t st, const TileConfig &tc) {
    if (total <= 0 || n_in <= 0) return GSMAT_OK;
    GS_TRY(tile_config_check(tc));
    const int items = tc.expand_items;
    const int64_t n_parts = (n_in + total + items - 1) / items;
    if (n_parts > INT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "expand into %lld rows", (long long)total);
    for (int c = 0; c <= k; ++c) {
        if (reinterpret_cast<uintptr_t>(out.c[c]) & 15u) {
            return set_error(GSMAT_ERR_INVALID_ARG, "expand output column %d not 16-byte aligned", c);
        }
    }
    DevBuf cuts;
    GS_TRY(cuts.alloc(sizeof(int64_t) * (size_t)(n_parts + 1), st));
    ExpandArgs a;
    a.items = items;
    a.val = sv.side[side].val;
    a.in = in;
    a.k = k;
    a.n_in = n_in;
    a.off = off;
    a.first = first;
    a.total = total;
    a.cuts = cuts.as<int64_t>();
    a.out = out;
    // algorithmic bytes (per the method): read k bound columns, the offset
    // and the first entry once per parent row, one neighbour id per output
    // row, write k + 1 columns per output row.
    KernelTimer t("expand", st, (double)n_in * (4.0 * k + 8.0 + 4.0) + (double)total * (4.0 + 4.0 * (k + 1)),
                  (double)total);
    static std::atomic<int> smem_set[64];
    const size_t smem = sizeof(int64_t) * (size_t)(items + 2) + sizeof(int32_t) * (size_t)(items + 1);
    GS_TRY(prepare_items_smem(expand_kernel, items, smem, smem_set));
    expand_partition_kernel<<<(unsigned)((n_parts + 1 + 255) / 256), 256, 0, st>>>(off, n_in, total, n_parts, items,
                                                                                  cuts.as<int64_t>());
    GS_LAUNCH_CHECK();
    expand_kernel<<<(unsigned)n_parts, kExBlock, smem, st>>>(a);
    GS_LAUNCH_CHECK();
    t.stop();
    return GSMAT_OK;
}

int launch_product_count_scan(const StoreView &sv, const ProdSpec &spec, const Cols &in, int64_t n, int64_t *off,
                              int32_t *first, int32_t *len, int64_t *d_total, int *err, cudaStream_t st) {
    if (n <= 0) {
        GS_CUDA(cudaMemsetAsync(off, 0, sizeof(int64_t), st));
        GS_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int64_t), st));
        return GSMAT_OK;
    }
    const int64_t ntiles = (n + kPcTile - 1) / kPcTile;
    if (ntiles > INT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "count over %lld rows", (long long)n);
    LookbackBuf lb;
    GS_TRY(lb.make(ntiles, st, err));
    // algorithmic bytes: per row factor the bound value, a row lookup and
    // the first entry and length out; the offset out
    KernelTimer t("product_count", st, (double)n * (8.0 + spec.nrow * (4.0 + 8.0 + 8.0)), (double)n);
    product_count_scan_kernel<<<(unsigned)ntiles, kPcBlock, 0, st>>>(sv, spec, in, n, off, first, len, d_total,
                                                                     lb.view);
    GS_LAUNCH_CHECK();
    t.stop();
    return GSMAT_OK;
}

static int product_out_cols(const ProdSpec &spec) {
    int c = 0;
    for (int i = 0; i < spec.nf; ++i) c += spec.f[i].kind == kProdPairs ? 2 : 1;
    return c;
}

int launch_product(const StoreView &sv, const ProdSpec &spec, const Cols &in, int k, int64_t n_in, const int64_t *off,
                   const int32_t *first, const int32_t *len, int64_t total, OutCols out, cudaStream_t st,
                   const TileConfig &tc) {
    if (total <= 0 || n_in <= 0) return GSMAT_OK;
    GS_TRY(tile_config_check(tc));
    const int items = tc.expand_items;
    if (total > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "product of %lld rows", (long long)total);
    for (int c = 0; c < k + product_out_cols(spec); ++c) {
        if (reinterpret_cast<uintptr_t>(out.c[c]) & 15u) {
            return set_error(GSMAT_ERR_INVALID_ARG, "product output column %d not 16-byte aligned", c);
        }
    }
    const int64_t n_parts = (n_in + total + items - 1) / items;
    DevBuf cuts;
    GS_TRY(cuts.alloc(sizeof(int64_t) * (size_t)(n_parts + 1), st));
    ProductArgs a;
    a.items = items;
    a.sv = sv;
    a.spec = spec;
    a.in = in;
    a.k = k;
    a.n_in = n_in;
    a.off = off;
    a.first = first;
    a.len = len;
    a.total = total;
    a.cuts = cuts.as<int64_t>();
    a.out = out;
    // algorithmic bytes: per input row its k columns, its offset and each
    // row factor's range; per output row the innermost factor's value read
    // and k + (factor columns) values written
    const int fc = product_out_cols(spec);
    KernelTimer t("product", st, (double)n_in * (4.0 * k + 8.0 + 8.0 * spec.nrow) + (double)total * (4.0 + 4.0 * (k + fc)),
                  (double)total);
    static std::atomic<int> smem_set[64];
    const size_t smem = sizeof(int64_t) * (size_t)(items + 2);
    GS_TRY(prepare_items_smem(product_kernel, items, smem, smem_set));
    expand_partition_kernel<<<(unsigned)((n_parts + 1 + 255) / 256), 256, 0, st>>>(off, n_in, total, n_parts, items,
                                                                                  cuts.as<int64_t>());
    GS_LAUNCH_CHECK();
    product_kernel<<<(unsigned)n_parts, kExBlock, smem, st>>>(a);
    GS_LAUNCH_CHECK();
    t.stop();
    return GSMAT_OK;
}

int launch_product_fixed(const ProdSpec &spec_in, int64_t total, OutCols out, cudaStream_t st) {
    if (total <= 0) return GSMAT_OK;
    if (total > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "product of %lld rows", (long long)total);
    ProdSpec spec = spec_in;
    uint64_t inner = 1;  // product of the lengths inside factor i (< 2^32: it divides total)
    for (int i = spec.nf - 1; i >= 0; --i) {
        spec.f[i].inner = make_fastdiv((uint32_t)inner);
        inner *= spec.f[i].len;
    }
    for (int c = 0; c < kMaxCols; ++c) {
        if (out.c[c] && (reinterpret_cast<uintptr_t>(out.c[c]) & 15u)) {
            return set_error(GSMAT_ERR_INVALID_ARG, "product output column %d not 16-byte aligned", c);
        }
    }
    const int fc = product_out_cols(spec);
    KernelTimer t("product", st, (double)total * (4.0 + 4.0 * fc), (double)total);
    int64_t g = (total / 4 + 255) / 256;
    if (g < 1) g = 1;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (g > cap) g = cap;
    product_fixed_kernel<<<(unsigned)g, 256, 0, st>>>(spec, (uint32_t)total, out);
    GS_LAUNCH_CHECK();
    t.stop();
    return GSMAT_OK;
}

int launch_filter(const StoreView &sv, const PredSide &ps_s, const PredSide &ps_o, ValueSrc s, ValueSrc o,
                  const Cols &in, int k, int64_t n_in, OutCols out, int64_t *d_count, int *err, cudaStream_t st,
                  const TileConfig &tc) {
    GS_TRY(tile_config_check(tc));
    FilterOp op;
    op.short_row = tc.short_row;
    op.s0 = sv.side[0];
    op.s1 = sv.side[1];
    op.ps_s = ps_s;
    op.ps_o = ps_o;
    op.s = s;
    op.o = o;
    op.in = in;
    op.k = k;
    op.out = out;
    // algorithmic bytes: the two tested columns, a row lookup and a probe
    // sector per row, plus reading and writing the surviving rows (counted at
    // the input size: an upper bound)
    KernelTimer t("filter", st, (double)n_in * (8.0 + 8.0 + 32.0 + 8.0 * k), (double)n_in);
    GS_TRY(run_select(op, n_in, d_count, st, err));
    t.stop();
    return GSMAT_OK;
}

int launch_isect_count(const StoreView &sv, int side_a, const PredSide &pa, ValueSrc a, int side_b, const PredSide &pb,
                       ValueSrc b, int64_t n, int32_t *counts, cudaStream_t st) {
    if (n <= 0) return GSMAT_OK;
    IsectSrc s{sv.side[side_a], sv.side[side_b], pa, pb, a, b};
    KernelTimer t("isect_count", st, (double)n * (8.0 + 16.0 + 4.0), (double)n);
    isect_count_kernel<<<grid_1d(n, 8), 256, 0, st>>>(s, n, counts);
    GS_LAUNCH_CHECK();
    t.stop();
    return GSMAT_OK;
}

int launch_isect_write(const StoreView &sv, int side_a, const PredSide &pa, ValueSrc a, int side_b, const PredSide &pb,
                       ValueSrc b, int64_t n, const int64_t *off, const Cols &in, int k, int64_t total, OutCols out,
                       cudaStream_t st) {
    if (n <= 0 || total <= 0) return GSMAT_OK;
    IsectSrc s{sv.side[side_a], sv.side[side_b], pa, pb, a, b};
    KernelTimer t("isect_write", st, (double)n * (8.0 + 16.0 + 8.0 + 4.0 * k) + (double)total * 4.0 * (k + 1),
                  (double)total);
    isect_write_kernel<<<grid_1d(n, 8), 256, 0, st>>>(s, n, off, in, k, out);
    GS_LAUNCH_CHECK();
    t.stop();
    return GSMAT_OK;
}

int launch_cross(const Cols &in, int k, int64_t n_in, const Cols &rel, int r_cols, int64_t m, OutCols out,
                 cudaStream_t st) {
    const uint64_t total = (uint64_t)n_in * (uint64_t)m;
    if (total == 0) return GSMAT_OK;
    if (total > UINT32_MAX || m > UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "cross product of %llu rows", (unsigned long long)total);
    KernelTimer t("cross", st, (double)total * 4.0 * (k + r_cols), (double)total);
    cross_kernel<<<grid_1d((int64_t)total, 256), 256, 0, st>>>(in, k, rel, r_cols, (uint32_t)m, total, out);
    GS_LAUNCH_CHECK();
    t.stop();
    return GSMAT_OK;
}

int launch_diag(const StoreView &sv, const PredSide &ps0, int32_t *out, int64_t *d_count, int *err, cudaStream_t st) {
    DiagOp op{sv.side[0].key + ps0.ent_base, sv.side[0].val + ps0.ent_base, out};
    return run_select(op, ps0.nnz, d_count, st, err);
}

int launch_const_lookup(const StoreView &sv, const PredSide *d_sides, int n_pred, const int32_t *d_req, int n_req,
                        int32_t *d_out, cudaStream_t st) {
    if (n_req <= 0) return GSMAT_OK;
    const_lookup_kernel<<<(n_req + 127) / 128, 128, 0, st>>>(sv, d_sides, n_pred, d_req, n_req, d_out);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

int launch_interleave(const Cols &in, int k, int64_t n, int32_t *dst, cudaStream_t st) {
    if (n <= 0 || k <= 0) return GSMAT_OK;
    interleave_kernel<<<grid_1d(n, 256), 256, 0, st>>>(in, k, n, dst);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

int launch_copy_cols(const Cols &in, int k, int64_t n, OutCols out, cudaStream_t st) {
    if (n <= 0 || k <= 0) return GSMAT_OK;
    copy_cols_kernel<<<grid_1d(n, 256), 256, 0, st>>>(in, k, n, out);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

}  // namespace gs
