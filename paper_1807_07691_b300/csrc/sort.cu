// Stable LSD radix sort of 32/64-bit keys with an optional 32- or 64-bit
// payload.
//
// Used by the store builder (sorting the triple set by (p, s, o) and
// (p, o, s), which lays out every predicate's matrix M_h of Sec. 5.3 row by
// row) and by the final canonical ordering of a result table.
//
// Onesweep structure: one histogram kernel counts the digits of every pass
// at once; then each 8-bit pass is a single kernel in which a CTA ranks one
// tile of keys stably (warp match_any on the digit, per-warp counters,
// cross-warp prefix), publishes its per-digit counts, finds the counts of
// all earlier tiles per digit by decoupled look-back (one thread per
// digit, bounded waits), stages the tile in shared memory in digit order
// and writes each digit's run to its global position.  Keys and payloads
// are read and written once per pass.
//
// The canonical reorder of a result table (reorder_rows) runs the same passes
// with the ends fused: the first pass packs each row's key from the table's
// columns itself and the last pass writes the sorted table's columns
// directly, so no key array is packed or unpacked separately.  The other
// columns reach the output one of three ways: carried through the passes as
// a packed 64-bit payload (when they fit it and are large), or gathered
// after the sort through the row index (the payload, or the key's low bits
// when index and key fit one word), column by column or as interleaved
// records.  Tables of at most 2048 rows are sorted by one CTA instead.
#include <atomic>

#include "common.cuh"
#include "join.cuh"

namespace gs {
namespace {

// Pass-kernel shape.  The defaults can be overridden at build time
// (-DGSMAT_PASS_MIN_BLOCKS=... and so on) to measure other shapes.
#ifndef GSMAT_PASS_MIN_BLOCKS
#define GSMAT_PASS_MIN_BLOCKS 4
#endif
#ifndef GSMAT_PASS_MIN_BLOCKS_KEYS
#define GSMAT_PASS_MIN_BLOCKS_KEYS 2  // 64-bit keys without a payload
#endif
#ifndef GSMAT_PASS_ITEMS_U64
#define GSMAT_PASS_ITEMS_U64 12
#endif
#ifndef GSMAT_PASS_ITEMS_U64_KEYS
#define GSMAT_PASS_ITEMS_U64_KEYS 24
#endif
#ifndef GSMAT_PASS_ITEMS_WIDE
#define GSMAT_PASS_ITEMS_WIDE 10
#endif
// How a warp finds the lanes whose key has its digit ("peers"): 1 from
// eight ballots, 2 by a shared-memory atomicOr of lane bits per digit, 0 by
// match_any.  Measured on B300: 2 is the fastest for 64-bit keys without a
// payload (8 % over 1), 1 for the rest (2-3 % over 2, 10 % over 0).
#ifndef GSMAT_RANK_KEYS
#define GSMAT_RANK_KEYS 2
#endif
#ifndef GSMAT_RANK_PAIRS
#define GSMAT_RANK_PAIRS 1
#endif
#ifndef GSMAT_RANK_PAIRWISE
#define GSMAT_RANK_PAIRWISE 1  // atomicOr ranking: two items per round, one mask table each
#endif
#ifndef GSMAT_LOOKBACK_WINDOW
#define GSMAT_LOOKBACK_WINDOW 8
#endif
// Sorts of 64-bit keys with a payload and at least GSMAT_BIG_SORT_N keys
// run a second pass shape: larger tiles at 2 CTAs per SM and the atomicOr
// ranking (about 8-14 % faster on 6x10^7 rows, slower on the small sorts,
// whose fewer tiles then underfill the GPU).
#ifndef GSMAT_BIG_SORT_N
#define GSMAT_BIG_SORT_N (1 << 23)
#endif
#ifndef GSMAT_PASS_ITEMS_U64_BIG
#define GSMAT_PASS_ITEMS_U64_BIG 20
#endif
#ifndef GSMAT_PASS_ITEMS_WIDE_BIG
#define GSMAT_PASS_ITEMS_WIDE_BIG 16
#endif
#ifndef GSMAT_PASS_MIN_BLOCKS_BIG
#define GSMAT_PASS_MIN_BLOCKS_BIG 2
#endif
#ifndef GSMAT_RANK_PAIRS_BIG
#define GSMAT_RANK_PAIRS_BIG 2
#endif
constexpr int kBlock = 256;               // histogram kernel
constexpr int kPassBlock = 256;           // pass kernel (a multiple of kBins)
constexpr int kPassWarps = kPassBlock / 32;
constexpr int kBins = 256;
constexpr int kMaxPasses = 8;
constexpr int kLookbackWindow = GSMAT_LOOKBACK_WINDOW;  // predecessor descriptors read per look-back round

template <class K>
struct SortTraits;
template <>
struct SortTraits<uint64_t> {
    static constexpr int kItems = GSMAT_PASS_ITEMS_U64;             // keys per thread with a payload
    static constexpr int kItemsKeysOnly = GSMAT_PASS_ITEMS_U64_KEYS; // and without
};
template <>
struct SortTraits<uint32_t> {
    static constexpr int kItems = 16;
    static constexpr int kItemsKeysOnly = 16;
};
// A 64-bit payload (packed column values carried through the passes)
// needs more registers and shared memory per key: fewer keys per thread.
// SHAPE 1: the large-sort shape (64-bit keys with a payload only).
template <class K, bool HasVals>
__host__ __device__ constexpr bool has_big_shape() {
    return HasVals && sizeof(K) == 8;
}
template <class K, bool HasVals, class V = uint32_t, int SHAPE = 0>
__host__ __device__ constexpr int items_per_thread() {
    return HasVals ? (sizeof(V) == 8 ? (SHAPE ? GSMAT_PASS_ITEMS_WIDE_BIG : GSMAT_PASS_ITEMS_WIDE)
                                     : (SHAPE ? GSMAT_PASS_ITEMS_U64_BIG : SortTraits<K>::kItems))
                   : SortTraits<K>::kItemsKeysOnly;
}

template <class K, bool HasVals, class V = uint32_t, int SHAPE = 0>
__host__ __device__ constexpr int rank_mode() {
    return (!HasVals && sizeof(K) == 8) ? GSMAT_RANK_KEYS : (SHAPE ? GSMAT_RANK_PAIRS_BIG : GSMAT_RANK_PAIRS);
}

// Pass CTAs resident per SM (the register budget of the launch bounds).
template <class K, bool HasVals, class V = uint32_t, int SHAPE = 0>
__host__ __device__ constexpr int pass_min_blocks() {
    return (!HasVals && sizeof(K) == 8) ? GSMAT_PASS_MIN_BLOCKS_KEYS
                                        : (SHAPE ? GSMAT_PASS_MIN_BLOCKS_BIG : GSMAT_PASS_MIN_BLOCKS);
}

template <class K>
__device__ __forceinline__ int digit_of(K k, int shift, int mask) {
    return (int)((k >> shift) & (K)mask);
}

// Tile descriptor of one digit: bits 56-63 pass epoch, 54-55 state, 0-53
// count.  A word whose epoch is not the current pass's is "not ready", so a
// single memset per sort serves every pass.
constexpr uint64_t kDescAggregate = 1;
constexpr uint64_t kDescPrefix = 2;
__device__ __forceinline__ unsigned long long desc_pack(uint32_t epoch, uint64_t state, uint64_t value) {
    return ((unsigned long long)epoch << 56) | (state << 54) | value;
}

// Key sources and sinks of a pass.  A source loads a thread's ITEMS keys and
// payloads of a tile (input positions t0 + base + 32 j, those below `valid`);
// a sink stores a sorted key and payload at position dst.
template <class K, bool HasVals, class V = uint32_t>
struct SrcArray {
    using Val = V;
    const K *keys;
    const V *vals;
    template <int ITEMS>
    __device__ __forceinline__ void load_tile(int64_t t0, int base, int valid, K (&k)[ITEMS], V (&v)[ITEMS]) const {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int idx = base + 32 * j;
            if (idx < valid) {
                k[j] = keys[t0 + idx];
                v[j] = HasVals ? vals[t0 + idx] : V(0);
            }
        }
    }
    // keys base + stride * j (those below n), all loads in flight together
    template <int H>
    __device__ __forceinline__ void hist_keys(int64_t base, int stride, int64_t n, K (&k)[H]) const {
#pragma unroll
        for (int j = 0; j < H; ++j) k[j] = base + (int64_t)stride * j < n ? __ldg(keys + base + (int64_t)stride * j) : K(0);
    }
};

// Rows of a column table: key = the fields of columns c[0..nc-1] of row r
// (most significant first, `bits` each), payload = r, where r = perm[i] (a
// permutation of 0..n-1) or i.  A tile's loads go column by column with all
// of a thread's rows in flight together.
//
// With idx_bits > 0 the row index rides in the key's low idx_bits bits
// instead of a separate payload (fields << idx_bits | r), so a pass moves 8
// bytes per row instead of 12; the passes then sort bits from idx_bits up.
struct SrcRows {
    using Val = uint32_t;
    const int32_t *c[kMaxCols];
    const uint32_t *perm;
    int nc;
    int bits;
    int idx_bits;
    template <int ITEMS>
    __device__ __forceinline__ void load_tile(int64_t t0, int base, int valid, uint64_t (&k)[ITEMS],
                                              uint32_t (&v)[ITEMS]) const {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int idx = base + 32 * j;
            v[j] = idx < valid ? (perm ? __ldg(perm + t0 + idx) : (uint32_t)(t0 + idx)) : 0u;
            k[j] = 0;
        }
        for (int cc = 0; cc < nc; ++cc) {
            const int32_t *col = c[cc];
            uint32_t x[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) x[j] = base + 32 * j < valid ? (uint32_t)__ldg(col + v[j]) : 0u;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) k[j] = (k[j] << bits) | x[j];
        }
        if (idx_bits) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) k[j] = (k[j] << idx_bits) | v[j];
        }
    }
    // digit counts do not depend on the order, so the histogram reads the
    // columns in place (fields only: pass p's digit is bits [8p, 8p + 8) of
    // the fields, at idx_bits + 8p in a packed key)
    template <int H>
    __device__ __forceinline__ void hist_keys(int64_t base, int stride, int64_t n, uint64_t (&k)[H]) const {
#pragma unroll
        for (int j = 0; j < H; ++j) k[j] = 0;
        for (int cc = 0; cc < nc; ++cc) {
            const int32_t *col = c[cc];
            uint32_t x[H];
#pragma unroll
            for (int j = 0; j < H; ++j) {
                const int64_t i = base + (int64_t)stride * j;
                x[j] = i < n ? (uint32_t)__ldg(col + i) : 0u;
            }
#pragma unroll
            for (int j = 0; j < H; ++j) k[j] = (k[j] << bits) | x[j];
        }
    }
};

template <class K, bool HasVals, class V = uint32_t>
struct SinkArray {
    K *keys;
    V *vals;
    __device__ __forceinline__ void store(uint32_t dst, K k, V v) const {
        keys[dst] = k;
        if (HasVals) vals[dst] = v;
    }
};

// Rows whose non-key columns travel with the key: key = the fields of
// columns c[0..nc-1], payload = the fields of columns c[nc..nc+nr-1] (nr *
// bits <= 64), both most significant first, `bits` each; rows in order.
struct SrcRowsWide {
    using Val = uint64_t;
    const int32_t *c[kMaxCols];
    int nc;
    int nr;
    int bits;
    template <int ITEMS>
    __device__ __forceinline__ void load_tile(int64_t t0, int base, int valid, uint64_t (&k)[ITEMS],
                                              uint64_t (&v)[ITEMS]) const {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            k[j] = 0;
            v[j] = 0;
        }
        for (int cc = 0; cc < nc + nr; ++cc) {
            const int32_t *col = c[cc];
            uint32_t x[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) x[j] = base + 32 * j < valid ? (uint32_t)__ldg(col + t0 + base + 32 * j) : 0u;
            if (cc < nc) {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) k[j] = (k[j] << bits) | x[j];
            } else {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) v[j] = (v[j] << bits) | x[j];
            }
        }
    }
    template <int H>
    __device__ __forceinline__ void hist_keys(int64_t base, int stride, int64_t n, uint64_t (&k)[H]) const {
#pragma unroll
        for (int j = 0; j < H; ++j) k[j] = 0;
        for (int cc = 0; cc < nc; ++cc) {
            const int32_t *col = c[cc];
            uint32_t x[H];
#pragma unroll
            for (int j = 0; j < H; ++j) {
                const int64_t i = base + (int64_t)stride * j;
                x[j] = i < n ? (uint32_t)__ldg(col + i) : 0u;
            }
#pragma unroll
            for (int j = 0; j < H; ++j) k[j] = (k[j] << bits) | x[j];
        }
    }
};

// The sorted table from key and payload alone: out[0..nc-1] from the key,
// out[nc..nc+nr-1] from the payload.
struct SinkRowsWide {
    int32_t *out[kMaxCols];
    int nc;
    int nr;
    int bits;
    __device__ __forceinline__ void store(uint32_t dst, uint64_t k, uint64_t v) const {
        const uint64_t fmask = (1ull << bits) - 1;
        for (int j = 0; j < nc; ++j) out[j][dst] = (int32_t)((k >> ((nc - 1 - j) * bits)) & fmask);
        for (int j = 0; j < nr; ++j) out[nc + j][dst] = (int32_t)((v >> ((nr - 1 - j) * bits)) & fmask);
    }
};

// Payload only (the permutation a later chunk starts from).
struct SinkPerm {
    uint32_t *vals;
    int idx_bits;  // > 0: the payload is the key's low idx_bits bits
    __device__ __forceinline__ void store(uint32_t dst, uint64_t k, uint32_t v) const {
        vals[dst] = idx_bits ? (uint32_t)(k & ((1ull << idx_bits) - 1)) : v;
    }
};

// The sorted table's leading columns: out[0..k0-1] unpacked from the key;
// the payload goes to perm (when not null) for the gather of the other
// columns, which runs as its own kernel at full occupancy.
struct SinkRows {
    int32_t *out[kMaxCols];
    uint32_t *perm;
    int k0;
    int bits;
    int idx_bits;  // > 0: the payload is the key's low idx_bits bits
    __device__ __forceinline__ void store(uint32_t dst, uint64_t k, uint32_t v) const {
        const uint64_t fmask = (1ull << bits) - 1;
        const uint64_t f = k >> idx_bits;
        for (int j = 0; j < k0; ++j) out[j][dst] = (int32_t)((f >> ((k0 - 1 - j) * bits)) & fmask);
        if (perm) perm[dst] = idx_bits ? (uint32_t)(k & ((1ull << idx_bits) - 1)) : v;
    }
};

// Gather of the non-key columns after the sort.  When consecutive output
// rows come from scattered input rows, reading each column costs one 32-byte
// sector per value; the columns are then first interleaved into records
// rec[i] = (rest[0][i], ..., rest[n_rest-1][i]) of rw int4 words
// (n_rest <= 4 * rw <= 8, zero padding), and the gather reads one sector per
// row.  When the permutation keeps runs of consecutive rows (trailing plan
// variables fan out inside each key group), the columns are read directly.
//
// *use_rec = 1 unless at least half of kLocalitySamples evenly spaced
// positions i have |perm[i + 1] - perm[i]| <= 8 (same or next sector).
constexpr int kLocalitySamples = 4096;
__global__ void __launch_bounds__(256) perm_locality_kernel(const uint32_t *__restrict__ perm, int64_t n,
                                                            int *__restrict__ use_rec) {
    __shared__ int64_t tmp[9];
    constexpr int kPer = kLocalitySamples / 256;
    uint32_t a[kPer], b[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int64_t k = threadIdx.x + 256 * u;
        const int64_t i = n > 1 ? k * (n - 2) / (kLocalitySamples - 1) : 0;
        a[u] = i + 1 < n ? __ldg(perm + i) : 0u;
        b[u] = i + 1 < n ? __ldg(perm + i + 1) : 0u;
    }
    int local = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int64_t d = (int64_t)b[u] - (int64_t)a[u];
        local += (n > 1 && d >= -8 && d <= 8) ? 1 : 0;
    }
    int64_t total;
    block_exclusive_sum<256>((int64_t)local, tmp, &total);
    if (threadIdx.x == 0) *use_rec = 2 * total < kLocalitySamples ? 1 : 0;
}

// Runs only when *use_rec is set (by perm_locality_kernel).
constexpr int kMaxRecCols = 8;
__global__ void __launch_bounds__(256) interleave_rest_kernel(Cols rest, int n_rest, int rw, int64_t n,
                                                              const int *__restrict__ use_rec,
                                                              int4 *__restrict__ rec) {
    if (!*use_rec) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int x[kMaxRecCols];
#pragma unroll
        for (int j = 0; j < kMaxRecCols; ++j) x[j] = j < n_rest ? __ldg(rest.c[j] + i) : 0;
        rec[i * rw] = make_int4(x[0], x[1], x[2], x[3]);
        if (rw > 1) rec[i * rw + 1] = make_int4(x[4], x[5], x[6], x[7]);
    }
}

// Each gather thread keeps kGatherRows rows' loads in flight.
constexpr int kGatherRows = 4;

// out[j][i] = rest[j][perm[i]], column by column.
__device__ __forceinline__ void gather_columns(const Cols &rest, const OutCols &out, int n_rest,
                                               const uint32_t *__restrict__ perm, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += stride * kGatherRows) {
        uint32_t r[kGatherRows];
#pragma unroll
        for (int u = 0; u < kGatherRows; ++u) {
            const int64_t i = i0 + u * stride;
            r[u] = i < n ? __ldg(perm + i) : 0u;
        }
        for (int j = 0; j < n_rest; ++j) {
            int32_t x[kGatherRows];
#pragma unroll
            for (int u = 0; u < kGatherRows; ++u) x[u] = i0 + u * stride < n ? __ldg(rest.c[j] + r[u]) : 0;
#pragma unroll
            for (int u = 0; u < kGatherRows; ++u) {
                if (i0 + u * stride < n) out.c[j][i0 + u * stride] = x[u];
            }
        }
    }
}

// out[j][i] = field j of rec[perm[i]]; runs only when *use_rec is set (the
// column gather runs otherwise, as its own kernel so that each keeps its
// own register budget and occupancy).
__global__ void __launch_bounds__(256) gather_rec_kernel(const int4 *__restrict__ rec, int rw,
                                                         const int *__restrict__ use_rec, int n_rest, OutCols out,
                                                         const uint32_t *__restrict__ perm, int64_t n) {
    if (!*use_rec) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += stride * kGatherRows) {
        int4 a[kGatherRows], b[kGatherRows];
#pragma unroll
        for (int u = 0; u < kGatherRows; ++u) {
            const int64_t i = i0 + u * stride;
            const uint32_t r = i < n ? __ldg(perm + i) : 0u;
            a[u] = i < n ? __ldg(rec + (int64_t)r * rw) : make_int4(0, 0, 0, 0);
            b[u] = (i < n && rw > 1) ? __ldg(rec + (int64_t)r * rw + 1) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < kGatherRows; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                const int x[kMaxRecCols] = {a[u].x, a[u].y, a[u].z, a[u].w, b[u].x, b[u].y, b[u].z, b[u].w};
#pragma unroll
                for (int j = 0; j < kMaxRecCols; ++j) {
                    if (j < n_rest) out.c[j][i] = x[j];
                }
            }
        }
    }
}

// Reorder of a small table (n <= kSmallSortRows, the m key columns packed
// in at most two 64-bit words) by one CTA: bitonic sort of (key, row) in
// shared memory (the row breaks ties, so the order is the stable one), then
// the output columns, key columns unpacked and the others gathered.
constexpr int kSmallSortRows = 2048;
constexpr int kSmallSortBlock = 1024;
__global__ void __launch_bounds__(kSmallSortBlock) small_reorder_kernel(Cols cols, int V, int m, int k0, int bits,
                                                                        int n, OutCols out) {
    __shared__ unsigned long long s0[kSmallSortRows], s1[kSmallSortRows];
    __shared__ uint16_t si[kSmallSortRows];
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int i = threadIdx.x; i < n2; i += kSmallSortBlock) {
        unsigned long long w0 = ~0ull, w1 = ~0ull;
        if (i < n) {
            w0 = 0;
            w1 = 0;
            for (int j = 0; j < k0; ++j) w0 = (w0 << bits) | (uint32_t)__ldg(cols.c[j] + i);
            for (int j = k0; j < m; ++j) w1 = (w1 << bits) | (uint32_t)__ldg(cols.c[j] + i);
        }
        s0[i] = w0;
        s1[i] = w1;
        si[i] = (uint16_t)(i < n ? i : 0xffff);
    }
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n2; i += kSmallSortBlock) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long ai = s0[i], aj = s0[j], bi = s1[i], bj = s1[j];
                    const uint16_t ii = si[i], ij = si[j];
                    const bool gt = ai > aj || (ai == aj && (bi > bj || (bi == bj && ii > ij)));
                    if (gt == up) {
                        s0[i] = aj;
                        s0[j] = ai;
                        s1[i] = bj;
                        s1[j] = bi;
                        si[i] = ij;
                        si[j] = ii;
                    }
                }
            }
            __syncthreads();
        }
    }
    const unsigned long long fmask = (1ull << bits) - 1;
    for (int i = threadIdx.x; i < n; i += kSmallSortBlock) {
        const int r = si[i];
        for (int j = 0; j < k0; ++j) out.c[j][i] = (int32_t)((s0[i] >> ((k0 - 1 - j) * bits)) & fmask);
        for (int j = k0; j < m; ++j) out.c[j][i] = (int32_t)((s1[i] >> ((m - 1 - j) * bits)) & fmask);
        for (int j = m; j < V; ++j) out.c[j][i] = __ldg(cols.c[j] + r);
    }
}

// The column gather; with use_rec given, runs only when *use_rec is clear.
__global__ void __launch_bounds__(256) gather_rest_kernel(Cols rest, OutCols out, int n_rest,
                                                          const uint32_t *__restrict__ perm, int64_t n,
                                                          const int *__restrict__ use_rec) {
    if (use_rec && *use_rec) return;
    gather_columns(rest, out, n_rest, perm, n);
}

// Digit counts of every pass in one read of the keys: CTA-wide shared
// histograms, each thread keeping kHistItems keys' loads in flight.  With
// kHistCopies > 1 lane l counts into copy l % kHistCopies, the copies a
// bank apart, so lanes with the same digit contend fewer ways on one word.
constexpr int kHistItems = 8;
#ifndef GSMAT_HIST_COPIES
#define GSMAT_HIST_COPIES 1
#endif
constexpr int kHistCopies = GSMAT_HIST_COPIES;
__host__ __device__ constexpr int hist_stride(int n_pass) { return n_pass * kBins + 1; }
template <class K, class Src>
__global__ void __launch_bounds__(kBlock) onesweep_histogram(Src src, int64_t n, int begin_bit, int end_bit,
                                                            int n_pass, uint32_t *__restrict__ hist) {
    extern __shared__ uint32_t hsm[];  // [kHistCopies][hist_stride(n_pass)]
    const int stride = hist_stride(n_pass);
    for (int i = threadIdx.x; i < kHistCopies * stride; i += kBlock) hsm[i] = 0;
    __syncthreads();
    uint32_t *mine = hsm + (threadIdx.x % kHistCopies) * stride;
    const int64_t span = (int64_t)kBlock * kHistItems;
    for (int64_t base = blockIdx.x * span + threadIdx.x; base < n; base += (int64_t)gridDim.x * span) {
        K k[kHistItems];
        src.template hist_keys<kHistItems>(base, kBlock, n, k);
#pragma unroll
        for (int j = 0; j < kHistItems; ++j) {
            if (base + (int64_t)kBlock * j < n) {
                for (int p = 0; p < n_pass; ++p) {
                    const int shift = begin_bit + 8 * p;
                    const int width = end_bit - shift < 8 ? end_bit - shift : 8;
                    atomicAdd(&mine[p * kBins + digit_of(k[j], shift, (1 << width) - 1)], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_pass * kBins; i += kBlock) {
        uint32_t c = 0;
#pragma unroll
        for (int cp = 0; cp < kHistCopies; ++cp) c += hsm[cp * stride + i];
        if (c) atomicAdd(hist + i, c);
    }
}

template <class K, bool HasVals, class Src, class Sink, int SHAPE = 0>
__global__ void __launch_bounds__(kPassBlock, (pass_min_blocks<K, HasVals, typename Src::Val, SHAPE>())) onesweep_pass(Src src, Sink sink, int64_t n, int shift, int mask,
                                                       const uint32_t *__restrict__ hist_pass,
                                                       unsigned long long *__restrict__ desc,
                                                       unsigned int *__restrict__ tile_counter, uint32_t epoch,
                                                       int *__restrict__ err) {
    using V = typename Src::Val;
    constexpr int ITEMS = items_per_thread<K, HasVals, V, SHAPE>();
    constexpr int TILE = kPassBlock * ITEMS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *skeys = reinterpret_cast<K *>(smem_raw);
    V *svals = reinterpret_cast<V *>(skeys + TILE);
    uint32_t *whist = reinterpret_cast<uint32_t *>(svals + (HasVals ? TILE : 0));  // [kPassWarps][kBins]
    uint32_t *gbase = whist + kPassWarps * kBins;
    constexpr int RANK = rank_mode<K, HasVals, V, SHAPE>();
    uint32_t *wmask = gbase + kBins;  // RANK 2: [kPassWarps][2][kBins] lane masks by digit
    __shared__ int64_t scan_tmp[kPassWarps + 1];
    __shared__ int tile_sm;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) tile_sm = (int)atomicAdd(tile_counter, 1u);
    for (int i = threadIdx.x; i < kPassWarps * kBins; i += kPassBlock) whist[i] = 0;
    if (RANK == 2) {
        for (int i = threadIdx.x; i < 2 * kPassWarps * kBins; i += kPassBlock) wmask[i] = 0;
    }
    __syncthreads();
    const int tile = tile_sm;
    const int64_t t0 = (int64_t)tile * TILE;
    const int valid = (int)((n - t0) < TILE ? (n - t0) : TILE);
    const unsigned lt_mask = (1u << lane) - 1u;
    uint32_t *wh = whist + warp * kBins;

    K k[ITEMS];
    V v[ITEMS];
    uint32_t dr[ITEMS];  // rank within the warp << 8 | digit
    // warp-striped: stable order inside the tile is (warp, j, lane)
    src.template load_tile<ITEMS>(t0, warp * (32 * ITEMS) + lane, valid, k, v);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int idx = warp * (32 * ITEMS) + j * 32 + lane;
        if (idx < valid) {
            dr[j] = (uint32_t)digit_of(k[j], shift, mask);
        } else {
            k[j] = ~K(0);
            v[j] = V(0);
            dr[j] = kBins - 1;  // padding ranks last in the last bucket
        }
    }
    if constexpr (RANK == 2 && GSMAT_RANK_PAIRWISE && ITEMS % 2 == 0) {
        // Two items per round, their lane bits in two tables, so the two
        // chains of shared-memory operations overlap.  Item j's counter
        // update is issued before item j + 1's, so equal digits keep the
        // order (j, lane).
        uint32_t *wa = wmask + warp * 2 * kBins, *wb = wa + kBins;
#pragma unroll
        for (int j = 0; j < ITEMS; j += 2) {
            const int d0 = (int)dr[j], d1 = (int)dr[j + 1];
            atomicOr(&wa[d0], 1u << lane);
            atomicOr(&wb[d1], 1u << lane);
            __syncwarp();
            const unsigned p0 = wa[d0], p1 = wb[d1];
            __syncwarp();
            if ((p0 & lt_mask) == 0) wa[d0] = 0;  // each leader clears its word for the next round
            if ((p1 & lt_mask) == 0) wb[d1] = 0;
            const int l0 = __ffs(p0) - 1, l1 = __ffs(p1) - 1;
            uint32_t b0 = 0, b1 = 0;
            if (lane == l0) b0 = atomicAdd(&wh[d0], (uint32_t)__popc(p0));
            if (lane == l1) b1 = atomicAdd(&wh[d1], (uint32_t)__popc(p1));
            b0 = __shfl_sync(0xffffffffu, b0, l0);
            b1 = __shfl_sync(0xffffffffu, b1, l1);
            dr[j] = ((b0 + (uint32_t)__popc(p0 & lt_mask)) << 8) | (uint32_t)d0;
            dr[j + 1] = ((b1 + (uint32_t)__popc(p1 & lt_mask)) << 8) | (uint32_t)d1;
            __syncwarp();
        }
    } else {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int d = (int)dr[j];
        unsigned peers;
        if (RANK == 2) {
            // every lane sets its bit in its digit's word; the word then holds the peers
            uint32_t *wm = wmask + warp * 2 * kBins;
            atomicOr(&wm[d], 1u << lane);
            __syncwarp();
            peers = wm[d];
            __syncwarp();
            if ((peers & lt_mask) == 0) wm[d] = 0;  // the leader clears it for the next round
        } else if (RANK == 1) {
            // lanes whose digit agrees with this lane's in every bit
            peers = 0xffffffffu;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const bool bit = (d >> b) & 1;
                const unsigned bal = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bal : ~bal;
            }
        } else {
            peers = __match_any_sync(0xffffffffu, d);
        }
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&wh[d], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        dr[j] = ((base + (uint32_t)__popc(peers & lt_mask)) << 8) | (uint32_t)d;
        __syncwarp();
    }
    }
    __syncthreads();
    // per digit (thread d < kBins): cross-warp prefix and the tile's count
    const int d = threadIdx.x;
    const bool dig = d < kBins;
    uint32_t cnt = 0;
    if (dig) {
#pragma unroll
        for (int w = 0; w < kPassWarps; ++w) {
            const uint32_t c = whist[w * kBins + d];
            whist[w * kBins + d] = cnt;
            cnt += c;
        }
    }
    const uint32_t real = cnt - (d == kBins - 1 ? (uint32_t)(TILE - valid) : 0u);
    // Publish this tile's count of digit d before anything else, so that
    // later tiles' look-backs find it as early as possible.  Tile 0
    // publishes its inclusive prefix instead, with the digit's global start
    // (exclusive scan of the pass histogram) folded in, so every later
    // tile's look-back sum is already a global position.
    int64_t tot;
    uint64_t excl = 0;
    if (tile == 0) {  // uniform over the CTA (the scan synchronises)
        const int64_t dbase =
            block_exclusive_sum<kPassBlock>(dig ? (int64_t)__ldg(hist_pass + d) : (int64_t)0, scan_tmp, &tot);
        excl = (uint64_t)dbase;
        if (dig) atomicExch(desc + d, desc_pack(epoch, kDescPrefix, excl + real));
    } else if (dig) {
        atomicExch(desc + (int64_t)tile * kBins + d, desc_pack(epoch, kDescAggregate, real));
    }
    // tile-local start of every digit, then the tile staged in shared memory
    // in digit order (the keys leave the registers before the look-back)
    // (each warp's counter of digit d becomes the staged position of its
    // first key of d: the digit's tile start plus the earlier warps' keys)
    const int64_t ts = block_exclusive_sum<kPassBlock>((int64_t)cnt, scan_tmp, &tot);
    if (dig) {
#pragma unroll
        for (int w = 0; w < kPassWarps; ++w) whist[w * kBins + d] += (uint32_t)ts;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t dd = dr[j] & 0xffu;
        const uint32_t pos = wh[dd] + (dr[j] >> 8);
        skeys[pos] = k[j];
        if (HasVals) svals[pos] = v[j];
    }
    // Look back for digit d over the earlier tiles, kLookbackWindow
    // descriptors in flight at a time (for each predecessor the CTA's 256
    // digit words are one contiguous 2 KB line set), summed nearest first up
    // to and including the first inclusive prefix.  A descriptor not yet
    // published stops the round; the next round starts from it.  The waits
    // are bounded: past kLookbackPollLimit the error word is set and the
    // missing counts are taken as zero.
    if (tile > 0 && dig) {
        int j = tile - 1;
        int polls = 0;
        while (true) {
            unsigned long long w[kLookbackWindow];
#pragma unroll
            for (int i = 0; i < kLookbackWindow; ++i) {
                w[i] = j - i >= 0 ? ld_volatile_u64(desc + (int64_t)(j - i) * kBins + d)
                                  : desc_pack(epoch, kDescPrefix, 0);
            }
            int used = 0;
            bool done = false, stalled = false;
#pragma unroll
            for (int i = 0; i < kLookbackWindow; ++i) {
                if (!done && !stalled) {
                    const uint64_t state = (w[i] >> 54) & 3;
                    if ((uint32_t)(w[i] >> 56) != epoch || state == 0) {
                        stalled = true;
                    } else {
                        excl += w[i] & ((1ull << 54) - 1);
                        used = i + 1;
                        done = state == kDescPrefix;
                    }
                }
            }
            if (done) break;
            j -= used;
            if (stalled) {
                if (++polls > kLookbackPollLimit) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        atomicExch(desc + (int64_t)tile * kBins + d, desc_pack(epoch, kDescPrefix, excl + real));
    }
    // global position of the tile's first key of digit d, minus that key's
    // place in the staged tile: key i of digit d goes to gdelta[d] + i
    if (dig) gbase[d] = (uint32_t)excl - (uint32_t)ts;
    __syncthreads();
    for (int i = threadIdx.x; i < valid; i += kPassBlock) {
        const K kk = skeys[i];
        const int dd = digit_of(kk, shift, mask);
        sink.store(gbase[dd] + (uint32_t)i, kk, HasVals ? svals[i] : V(0));
    }
}

int sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int v = cached[dev].load(std::memory_order_acquire);
    if (!v) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 148;
        }
        cached[dev].store(v, std::memory_order_release);
    }
    return v;
}

template <class K, bool HasVals, class V, int SHAPE = 0>
int pass_smem_bytes() {
    constexpr int TILE = kPassBlock * items_per_thread<K, HasVals, V, SHAPE>();
    return TILE * (int)sizeof(K) + (HasVals ? TILE * (int)sizeof(V) : 0) +
           (kPassWarps * kBins * (rank_mode<K, HasVals, V, SHAPE>() == 2 ? 3 : 1) + kBins) * 4;
}

int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return (dev < 0 || dev >= 64) ? 0 : dev;
}

template <class K, bool HasVals, class Src, class Sink, int SHAPE>
int launch_pass_shape(const Src &src, const Sink &sink, int64_t n, int shift, int width, const uint32_t *hist_pass,
                      unsigned long long *desc, unsigned int *counter, uint32_t epoch, int *err, cudaStream_t st) {
    using V = typename Src::Val;
    static std::atomic<bool> done[64];  // attributes set (once per device; setting them twice is harmless)
    const int dev = current_device();
    if (!done[dev].load(std::memory_order_acquire)) {
        GS_CUDA(cudaFuncSetAttribute(onesweep_pass<K, HasVals, Src, Sink, SHAPE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     pass_smem_bytes<K, HasVals, V, SHAPE>()));
        // the driver's own carveout: forcing the maximum shared memory left
        // too little L1 for the passes that gather through a permutation
        GS_CUDA(cudaFuncSetAttribute(onesweep_pass<K, HasVals, Src, Sink, SHAPE>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutDefault));
        done[dev].store(true, std::memory_order_release);
    }
    constexpr int TILE = kPassBlock * items_per_thread<K, HasVals, V, SHAPE>();
    const int64_t ntiles = (n + TILE - 1) / TILE;
    onesweep_pass<K, HasVals, Src, Sink, SHAPE>
        <<<(unsigned)ntiles, kPassBlock, pass_smem_bytes<K, HasVals, V, SHAPE>(), st>>>(
            src, sink, n, shift, (1 << width) - 1, hist_pass, desc, counter, epoch, err);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

// One pass; its descriptors were sized for the default shape's tiles (the
// large-sort shape's tiles are larger, so they need fewer).
template <class K, bool HasVals, class Src, class Sink>
int launch_pass(const Src &src, const Sink &sink, int64_t n, int shift, int width, const uint32_t *hist_pass,
                unsigned long long *desc, unsigned int *counter, uint32_t epoch, int *err, cudaStream_t st) {
    if constexpr (has_big_shape<K, HasVals>()) {
        if (n >= (int64_t)GSMAT_BIG_SORT_N) {
            return launch_pass_shape<K, HasVals, Src, Sink, 1>(src, sink, n, shift, width, hist_pass, desc, counter,
                                                               epoch, err, st);
        }
    }
    return launch_pass_shape<K, HasVals, Src, Sink, 0>(src, sink, n, shift, width, hist_pass, desc, counter, epoch,
                                                       err, st);
}

template <class K, class Src>
int launch_histogram(const Src &src, int64_t n, int begin_bit, int end_bit, int n_pass, uint32_t *hist,
                     cudaStream_t st) {
    const int64_t span = (int64_t)kBlock * kHistItems;
    int64_t g = (n + span - 1) / span;
    const int smem = kHistCopies * hist_stride(n_pass) * (int)sizeof(uint32_t);
    const int64_t per_sm = std::max(1, std::min(8, (200 * 1024) / smem));  // resident CTAs
    const int64_t cap = (int64_t)sm_count() * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    if (smem > 48 * 1024) {
        static std::atomic<bool> done[64];  // attribute set (once per device)
        const int dev = current_device();
        if (!done[dev].load(std::memory_order_acquire)) {
            GS_CUDA(cudaFuncSetAttribute(onesweep_histogram<K, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kHistCopies * hist_stride(kMaxPasses) * (int)sizeof(uint32_t)));
            done[dev].store(true, std::memory_order_release);
        }
    }
    onesweep_histogram<K, Src><<<(unsigned)g, kBlock, smem, st>>>(src, n, begin_bit, end_bit, n_pass, hist);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

// Per-sort scratch: digit histograms | tile counters | error word | tile
// descriptors, zeroed by one memset.
struct SortMeta {
    DevBuf buf;
    uint32_t *hist = nullptr;
    unsigned int *counters = nullptr;
    int *err = nullptr;
    unsigned long long *desc = nullptr;

    int make(int64_t n, int n_pass, int tile, cudaStream_t st, int *err_word) {
        const int64_t ntiles = (n + tile - 1) / tile;
        const size_t off_cnt = round_up(sizeof(uint32_t) * kBins * n_pass, 256);
        const size_t off_err = off_cnt + sizeof(uint32_t) * kMaxPasses;
        const size_t off_desc = round_up(off_err + sizeof(int), 256);
        const size_t bytes = off_desc + sizeof(unsigned long long) * kBins * (size_t)ntiles;
        GS_TRY(buf.alloc(bytes, st));
        GS_CUDA(cudaMemsetAsync(buf.p, 0, bytes, st));
        hist = buf.as<uint32_t>();
        counters = reinterpret_cast<unsigned int *>(buf.as<char>() + off_cnt);
        err = err_word ? err_word : reinterpret_cast<int *>(buf.as<char>() + off_err);
        desc = reinterpret_cast<unsigned long long *>(buf.as<char>() + off_desc);
        return GSMAT_OK;
    }
};

// With alt_keys given, it is the second key buffer (nothing allocated for
// it) and *sorted_out receives whichever buffer holds the result (no copy
// back); otherwise the result is copied back into keys / vals.
template <class K, bool HasVals, class V = uint32_t>
int sort_passes(K *keys, V *vals, int64_t n, int begin_bit, int end_bit, cudaStream_t st, int *err_word,
                K *alt_keys = nullptr, K **sorted_out = nullptr) {
    using SA = SrcArray<K, HasVals, V>;
    using KA = SinkArray<K, HasVals, V>;
    const int n_pass = (end_bit - begin_bit + 7) / 8;
    SortMeta meta;
    GS_TRY(meta.make(n, n_pass, kPassBlock * items_per_thread<K, HasVals, V>(), st, err_word));
    DevBuf alt_k, alt_v;
    if (!alt_keys) GS_TRY(alt_k.alloc(sizeof(K) * (size_t)n, st));
    if (HasVals) GS_TRY(alt_v.alloc(sizeof(V) * (size_t)n, st));
    GS_TRY((launch_histogram<K, SA>(SA{keys, vals}, n, begin_bit, end_bit, n_pass, meta.hist, st)));
    K *src_k = keys, *dst_k = alt_keys ? alt_keys : alt_k.as<K>();
    V *src_v = vals, *dst_v = alt_v.as<V>();
    for (int p = 0; p < n_pass; ++p) {
        const int shift = begin_bit + 8 * p;
        const int width = end_bit - shift < 8 ? end_bit - shift : 8;
        GS_TRY((launch_pass<K, HasVals, SA, KA>(SA{src_k, src_v}, KA{dst_k, dst_v}, n, shift, width,
                                               meta.hist + p * kBins, meta.desc, meta.counters + p, (uint32_t)(p + 1),
                                               meta.err, st)));
        K *tk = src_k; src_k = dst_k; dst_k = tk;
        V *tv = src_v; src_v = dst_v; dst_v = tv;
    }
    if (sorted_out) {
        *sorted_out = src_k;
    } else if (src_k != keys) {
        GS_CUDA(cudaMemcpyAsync(keys, src_k, sizeof(K) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        if (HasVals) GS_CUDA(cudaMemcpyAsync(vals, src_v, sizeof(V) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    }
    return GSMAT_OK;
}

template <class K>
int radix_sort_impl(K *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit, cudaStream_t st,
                    const char *timer_name, int *err_word) {
    if (n < 0) return set_error(GSMAT_ERR_INVALID_ARG, "radix sort: negative n");
    if (begin_bit < 0 || end_bit > (int)(8 * sizeof(K)) || begin_bit > end_bit) {
        return set_error(GSMAT_ERR_INVALID_ARG, "radix sort: bad bit range [%d,%d)", begin_bit, end_bit);
    }
    if (n <= 1 || begin_bit == end_bit) return GSMAT_OK;
    if (n > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "radix sort: n = %lld >= 2^32", (long long)n);
    const int n_pass = (end_bit - begin_bit + 7) / 8;
    KernelTimer t(timer_name, st, (double)n * (2.0 * sizeof(K) + (vals ? 8.0 : 0.0)) * n_pass, (double)n);
    const int rc = vals ? sort_passes<K, true>(keys, vals, n, begin_bit, end_bit, st, err_word)
                        : sort_passes<K, false>(keys, static_cast<uint32_t *>(nullptr), n, begin_bit, end_bit, st,
                                                err_word);
    if (rc != GSMAT_OK) return rc;
    t.stop();
    return GSMAT_OK;
}

// One pass of a row sort, with the source and sink the pass's place calls for.
template <bool HasVals>
int row_pass(bool first, bool last, bool final_chunk, const SrcRows &rows, const SinkRows &out, const SinkPerm &perm,
             const uint64_t *sk, const uint32_t *sv, uint64_t *dk, uint32_t *dv, int64_t n, int shift, int width,
             const uint32_t *hist_pass, unsigned long long *desc, unsigned int *counter, uint32_t epoch, int *err,
             cudaStream_t st) {
    using SA = SrcArray<uint64_t, HasVals>;
    using KA = SinkArray<uint64_t, HasVals>;
    const SA arr{sk, sv};
    const KA to{dk, dv};
    if (first && last) {
        return final_chunk ? launch_pass<uint64_t, HasVals, SrcRows, SinkRows>(rows, out, n, shift, width, hist_pass,
                                                                               desc, counter, epoch, err, st)
                           : launch_pass<uint64_t, HasVals, SrcRows, SinkPerm>(rows, perm, n, shift, width, hist_pass,
                                                                               desc, counter, epoch, err, st);
    }
    if (first) {
        return launch_pass<uint64_t, HasVals, SrcRows, KA>(rows, to, n, shift, width, hist_pass, desc, counter, epoch,
                                                           err, st);
    }
    if (last) {
        return final_chunk ? launch_pass<uint64_t, HasVals, SA, SinkRows>(arr, out, n, shift, width, hist_pass, desc,
                                                                          counter, epoch, err, st)
                           : launch_pass<uint64_t, HasVals, SA, SinkPerm>(arr, perm, n, shift, width, hist_pass, desc,
                                                                          counter, epoch, err, st);
    }
    return launch_pass<uint64_t, HasVals, SA, KA>(arr, to, n, shift, width, hist_pass, desc, counter, epoch, err, st);
}

}  // namespace

int radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit, cudaStream_t st,
                   int *err_word) {
    return radix_sort_impl<uint64_t>(keys, vals, n, begin_bit, end_bit, st, "radix_sort_u64", err_word);
}

int radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit, cudaStream_t st,
                   int *err_word) {
    return radix_sort_impl<uint32_t>(keys, vals, n, begin_bit, end_bit, st, "radix_sort_u32", err_word);
}

int radix_sort_u64_pingpong(uint64_t *keys, uint64_t *alt, int64_t n, int begin_bit, int end_bit, cudaStream_t st,
                            int *err_word, uint64_t **sorted) {
    if (n < 0 || !sorted || begin_bit < 0 || end_bit > 64 || begin_bit > end_bit) {
        return set_error(GSMAT_ERR_INVALID_ARG, "radix sort: bad arguments");
    }
    *sorted = keys;
    if (n <= 1 || begin_bit == end_bit) return GSMAT_OK;
    if (n > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "radix sort: n = %lld >= 2^32", (long long)n);
    const int n_pass = (end_bit - begin_bit + 7) / 8;
    KernelTimer t("radix_sort_u64", st, (double)n * 16.0 * n_pass, (double)n);
    GS_TRY((sort_passes<uint64_t, false>(keys, static_cast<uint32_t *>(nullptr), n, begin_bit, end_bit, st, err_word,
                                         alt, sorted)));
    t.stop();
    return GSMAT_OK;
}

int radix_sort_u64_wide(uint64_t *keys, uint64_t *vals, int64_t n, int begin_bit, int end_bit, cudaStream_t st,
                        int *err_word) {
    if (n < 0 || begin_bit < 0 || end_bit > 64 || begin_bit > end_bit || !vals) {
        return set_error(GSMAT_ERR_INVALID_ARG, "radix sort: bad arguments");
    }
    if (n <= 1 || begin_bit == end_bit) return GSMAT_OK;
    if (n > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "radix sort: n = %lld >= 2^32", (long long)n);
    const int n_pass = (end_bit - begin_bit + 7) / 8;
    KernelTimer t("radix_sort_u64", st, (double)n * 32.0 * n_pass, (double)n);
    GS_TRY((sort_passes<uint64_t, true, uint64_t>(keys, vals, n, begin_bit, end_bit, st, err_word)));
    t.stop();
    return GSMAT_OK;
}

namespace {

constexpr double kWideMinRestBytes = 256.0 * (1 << 20);

// Single-chunk reorder whose n_rest non-key columns fit one 64-bit payload:
// they travel through the passes with the key, so the sorted table comes
// out of the last pass whole (no permutation, no gather).
int reorder_wide(const Cols &cols, int V, int m, int bits, int64_t n, const OutCols &out, cudaStream_t st,
                 int *err_word) {
    using SA = SrcArray<uint64_t, true, uint64_t>;
    using KA = SinkArray<uint64_t, true, uint64_t>;
    const int n_rest = V - m;
    const int key_bits = m * bits;
    const int n_pass = (key_bits + 7) / 8;
    SrcRowsWide src;
    SinkRowsWide sink;
    memset(&src, 0, sizeof(src));
    memset(&sink, 0, sizeof(sink));
    for (int v = 0; v < V; ++v) {
        src.c[v] = cols.c[v];
        sink.out[v] = out.c[v];
    }
    src.nc = sink.nc = m;
    src.nr = sink.nr = n_rest;
    src.bits = sink.bits = bits;
    // algorithmic bytes: histogram 4m, first pass reads 4V, each pass
    // boundary writes and reads 16 (key + payload), last pass writes 4V
    const double algo = 4.0 * m + 8.0 * V + 32.0 * (n_pass - 1);
    KernelTimer t("reorder_sort", st, algo * (double)n, (double)n);
    DevBuf ka, kb, va, vb;
    GS_TRY(ka.alloc(sizeof(uint64_t) * (size_t)n, st));
    GS_TRY(va.alloc(sizeof(uint64_t) * (size_t)n, st));
    if (n_pass > 2) {
        GS_TRY(kb.alloc(sizeof(uint64_t) * (size_t)n, st));
        GS_TRY(vb.alloc(sizeof(uint64_t) * (size_t)n, st));
    }
    SortMeta meta;
    GS_TRY(meta.make(n, n_pass, kPassBlock * items_per_thread<uint64_t, true, uint64_t>(), st, err_word));
    GS_TRY((launch_histogram<uint64_t, SrcRowsWide>(src, n, 0, key_bits, n_pass, meta.hist, st)));
    for (int p = 0; p < n_pass; ++p) {
        const int shift = 8 * p;
        const int width = key_bits - shift < 8 ? key_bits - shift : 8;
        // pass p writes buffer set p & 1 and reads set (p - 1) & 1
        uint64_t *dk = (p & 1) ? kb.as<uint64_t>() : ka.as<uint64_t>();
        uint64_t *dv = (p & 1) ? vb.as<uint64_t>() : va.as<uint64_t>();
        const SA arr{(p & 1) ? ka.as<uint64_t>() : kb.as<uint64_t>(), (p & 1) ? va.as<uint64_t>() : vb.as<uint64_t>()};
        const KA to{dk, dv};
        const bool first = p == 0, last = p == n_pass - 1;
        const uint32_t *hp = meta.hist + p * kBins;
        unsigned int *ctr = meta.counters + p;
        const uint32_t ep = (uint32_t)(p + 1);
        if (first && last) {
            GS_TRY((launch_pass<uint64_t, true, SrcRowsWide, SinkRowsWide>(src, sink, n, shift, width, hp, meta.desc,
                                                                          ctr, ep, meta.err, st)));
        } else if (first) {
            GS_TRY((launch_pass<uint64_t, true, SrcRowsWide, KA>(src, to, n, shift, width, hp, meta.desc, ctr, ep,
                                                                meta.err, st)));
        } else if (last) {
            GS_TRY((launch_pass<uint64_t, true, SA, SinkRowsWide>(arr, sink, n, shift, width, hp, meta.desc, ctr, ep,
                                                                 meta.err, st)));
        } else {
            GS_TRY((launch_pass<uint64_t, true, SA, KA>(arr, to, n, shift, width, hp, meta.desc, ctr, ep, meta.err,
                                                       st)));
        }
    }
    t.stop();
    return GSMAT_OK;
}

}  // namespace

int reorder_rows(const Cols &cols, int V, int m, int bits, int64_t n, const OutCols &out, cudaStream_t st,
                 int *err_word, int mode) {
    if (V < 1 || V > kMaxCols || m < 1 || m > V || bits < 1 || bits > 31 || n < 0) {
        return set_error(GSMAT_ERR_INVALID_ARG, "reorder: V=%d m=%d bits=%d n=%lld", V, m, bits, (long long)n);
    }
    if (n == 0) return GSMAT_OK;
    if (n > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "reorder: n = %lld >= 2^32", (long long)n);
    const int per_key = 64 / bits;
    const int n_chunks = (m + per_key - 1) / per_key;
    const int k0 = m < per_key ? m : per_key;
    // Carrying the non-key columns costs 8 more bytes per row each way per
    // pass; a gather after the sort costs one random access per row, cheap
    // while the gathered columns stay in L2 (126 MB).  Carry them when they
    // fit 64 bits, the key needs at most five passes and the columns are
    // well beyond L2 (measured: 62 M rows x 3 columns, 5 passes, 11 % faster;
    // 12 M x 3 and 18 M x 2 with 8 passes, slower).
    const int n_pass_key = (m * bits + 7) / 8;
    const bool can_carry = n > kSmallSortRows && n_chunks == 1 && V > m && (V - m) * bits <= 64;
    const bool carry = mode == kReorderCarry ||
                       (mode == kReorderAuto && n_pass_key <= 5 && (double)n * (V - m) * 4.0 > kWideMinRestBytes);
    if (can_carry && carry) {
        return reorder_wide(cols, V, m, bits, n, out, st, err_word);
    }
    if (n <= kSmallSortRows && n_chunks <= 2) {
        KernelTimer t("reorder_sort", st, (8.0 * V) * (double)n, (double)n);
        small_reorder_kernel<<<1, kSmallSortBlock, 0, st>>>(cols, V, m, k0, bits, (int)n, out);
        GS_LAUNCH_CHECK();
        t.stop();
        return GSMAT_OK;
    }
    DevBuf ka, kb, va, vb, pa, pb;
    GS_TRY(ka.alloc(sizeof(uint64_t) * (size_t)n, st));
    GS_TRY(kb.alloc(sizeof(uint64_t) * (size_t)n, st));
    GS_TRY(va.alloc(sizeof(uint32_t) * (size_t)n, st));
    GS_TRY(vb.alloc(sizeof(uint32_t) * (size_t)n, st));
    if (n_chunks > 1) {
        GS_TRY(pa.alloc(sizeof(uint32_t) * (size_t)n, st));
        GS_TRY(pb.alloc(sizeof(uint32_t) * (size_t)n, st));
    }
    const int n_rest = V - k0;
    // row index width for keys that carry it in their low bits
    const int idx_bits = std::max(1, bits_for((uint64_t)(n - 1)));
    // algorithmic bytes: the histogram reads the key columns; the first pass
    // reads them (and the previous chunk's permutation); the last writes the
    // permutation, or the k0 leading output columns and (when other columns
    // follow) the payload, which the gather reads back with the n_rest
    // gathered values and writes n_rest columns; every other transfer is a
    // key and a payload
    double algo = n_rest > 0 ? 4.0 + 8.0 * n_rest : 0.0;
    for (int ci = n_chunks - 1; ci >= 0; --ci) {
        const int nc = (ci * per_key + per_key < m ? per_key : m - ci * per_key);
        const int n_pass = (nc * bits + 7) / 8;
        const double e = nc * bits + idx_bits <= 64 ? 8.0 : 12.0;  // bytes of one row between passes
        const double in0 = 4.0 * nc + (ci < n_chunks - 1 ? 4.0 : 0.0);
        const double outl = ci == 0 ? 4.0 * k0 + (n_rest > 0 ? 4.0 : 0.0) : 4.0;
        algo += 4.0 * nc + in0 + outl + (n_pass > 1 ? 2.0 * e : 0.0) + 2.0 * e * (n_pass > 2 ? n_pass - 2 : 0);
    }
    KernelTimer t("reorder_sort", st, algo * (double)n, (double)n);
    // the columns gathered after the sort, as records when they fit one
    Cols rest;
    OutCols ro;
    memset(&rest, 0, sizeof(rest));
    memset(&ro, 0, sizeof(ro));
    for (int j = 0; j < n_rest; ++j) {
        rest.c[j] = cols.c[k0 + j];
        ro.c[j] = out.c[k0 + j];
    }
    const int rw = n_rest == 0 ? 0 : (n_rest <= 4 ? 1 : (n_rest <= kMaxRecCols ? 2 : 0));
    const uint32_t *perm_in = nullptr;
    const uint32_t *final_perm = nullptr;
    for (int ci = n_chunks - 1; ci >= 0; --ci) {
        const int b = ci * per_key;
        const int e = m < b + per_key ? m : b + per_key;
        const int nc = e - b;
        const int key_bits = nc * bits;
        const int n_pass = (key_bits + 7) / 8;
        SrcRows src;
        memset(&src, 0, sizeof(src));
        for (int j = 0; j < nc; ++j) src.c[j] = cols.c[b + j];
        src.perm = perm_in;
        src.nc = nc;
        src.bits = bits;
        const bool packed = key_bits + idx_bits <= 64;
        src.idx_bits = packed ? idx_bits : 0;
        uint32_t *pout = ((n_chunks - 1 - ci) & 1) ? pb.as<uint32_t>() : pa.as<uint32_t>();
        const SinkPerm sink_perm{pout, src.idx_bits};
        SortMeta meta;
        GS_TRY(meta.make(n, n_pass,
                         kPassBlock * (packed ? items_per_thread<uint64_t, false>() : items_per_thread<uint64_t, true>()),
                         st, err_word));
        GS_TRY((launch_histogram<uint64_t, SrcRows>(src, n, 0, key_bits, n_pass, meta.hist, st)));
        for (int p = 0; p < n_pass; ++p) {
            const int shift = src.idx_bits + 8 * p;
            const int width = key_bits - 8 * p < 8 ? key_bits - 8 * p : 8;
            // pass p writes buffer set p & 1 and reads set (p - 1) & 1 (the
            // last pass of the final chunk writes the output columns and
            // its payload into set p & 1, which nothing reads then)
            uint64_t *dk = (p & 1) ? kb.as<uint64_t>() : ka.as<uint64_t>();
            uint32_t *dv = (p & 1) ? vb.as<uint32_t>() : va.as<uint32_t>();
            const uint64_t *sk = (p & 1) ? ka.as<uint64_t>() : kb.as<uint64_t>();
            const uint32_t *sv = (p & 1) ? va.as<uint32_t>() : vb.as<uint32_t>();
            SinkRows sink_rows;
            memset(&sink_rows, 0, sizeof(sink_rows));
            for (int v = 0; v < k0; ++v) sink_rows.out[v] = out.c[v];
            sink_rows.perm = n_rest > 0 ? dv : nullptr;
            sink_rows.k0 = k0;
            sink_rows.bits = bits;
            sink_rows.idx_bits = src.idx_bits;
            if (ci == 0 && p == n_pass - 1) final_perm = sink_rows.perm;
            if (packed) {
                GS_TRY(row_pass<false>(p == 0, p == n_pass - 1, ci == 0, src, sink_rows, sink_perm, sk, nullptr, dk,
                                       nullptr, n, shift, width, meta.hist + p * kBins, meta.desc, meta.counters + p,
                                       (uint32_t)(p + 1), meta.err, st));
            } else {
                GS_TRY(row_pass<true>(p == 0, p == n_pass - 1, ci == 0, src, sink_rows, sink_perm, sk, sv, dk, dv, n,
                                      shift, width, meta.hist + p * kBins, meta.desc, meta.counters + p,
                                      (uint32_t)(p + 1), meta.err, st));
            }
        }
        perm_in = pout;
    }
    if (n_rest > 0) {
        int64_t g = (n + 256 * kGatherRows - 1) / (256 * kGatherRows);
        const int64_t cap = (int64_t)sm_count() * 8;
        if (g > cap) g = cap;
        if (rw > 0) {
            DevBuf rec, flag;
            GS_TRY(rec.alloc(sizeof(int4) * (size_t)rw * (size_t)n, st));
            GS_TRY(flag.alloc(sizeof(int), st));
            perm_locality_kernel<<<1, 256, 0, st>>>(final_perm, n, flag.as<int>());
            GS_LAUNCH_CHECK();
            interleave_rest_kernel<<<grid_1d(n, 256), 256, 0, st>>>(rest, n_rest, rw, n, flag.as<int>(), rec.as<int4>());
            GS_LAUNCH_CHECK();
            gather_rec_kernel<<<(unsigned)g, 256, 0, st>>>(rec.as<int4>(), rw, flag.as<int>(), n_rest, ro, final_perm,
                                                           n);
            GS_LAUNCH_CHECK();
            gather_rest_kernel<<<(unsigned)g, 256, 0, st>>>(rest, ro, n_rest, final_perm, n, flag.as<int>());
        } else {
            gather_rest_kernel<<<(unsigned)g, 256, 0, st>>>(rest, ro, n_rest, final_perm, n, nullptr);
        }
        GS_LAUNCH_CHECK();
    }
    t.stop();
    return GSMAT_OK;
}

int device_sm_count() { return sm_count(); }

}  // namespace gs
