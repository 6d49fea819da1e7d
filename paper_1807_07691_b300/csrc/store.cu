// Device storage builder (Sec. 5): from an int32 (s, p, o) triple multiset
// to the per-predicate sparse matrices M_h, stored on both sides.
//
// Steps (Sec. 5.1 lists the paper's three: encode, build the cube, store
// the cube per predicate with statistics; ids arrive already encoded):
//  1. validate ids and find their ranges;
//  2. the distinct predicates (radix sort + unique) -> predicate slots and
//     the predicate hash index (host and device copies);
//  3. sort the triples by (slot, s, o), drop repeats (a dataset is a set,
//     Sec. 3.1) -> side 0 entries;
//  4. sort the unique triples by (slot, o, s) -> side 1 entries;
//  5. per side: non-zero rows (id, first entry) = the auxiliary arrays Row /
//     Rpos of Sec. 6.3, per predicate its first entry, nnz (the statistic m)
//     and first row; dense row pointers for predicates with many entries.
#include <string.h>

#include <algorithm>

#include "select.cuh"
#include "store.cuh"

namespace gs {

uint32_t pred_hash(int32_t p) { return (uint32_t)p * 2654435761u; }

namespace {

constexpr int kThreads = 256;

unsigned grid_for(int64_t n) { return grid_1d(n, kThreads); }

// ranges[0..3] = max subject/object, max predicate, min id, predicate
// overflow flag; ranges[4..4 + kPredTable) = open-addressing set of the
// predicates present (-1 = empty).  Each CTA first collects its predicates
// in a shared-memory set (a plain read finds those already there, so the
// loop issues almost no atomics), then inserts them into the global set.
// More distinct predicates than a set holds set the flag; the distinct
// predicates are then found by sorting.
constexpr int kPredLocal = 1024;
constexpr int kPredTable = 4096;
constexpr int kRangesWords = 4 + kPredTable;

__device__ __forceinline__ uint32_t pred_slot_hash(int32_t p) { return (uint32_t)p * 2654435761u; }

// Inserts p into the set table[0..cap) (cap a power of two); false if full.
__device__ __forceinline__ bool set_insert(int *table, int cap, int32_t p) {
    uint32_t h = pred_slot_hash(p) & (uint32_t)(cap - 1);
    for (int probe = 0; probe < cap; ++probe) {
        const int v = *(volatile int *)(table + h);
        if (v == p) return true;
        if (v == -1) {
            const int old = atomicCAS(table + h, -1, p);
            if (old == -1 || old == p) return true;
        }
        h = (h + 1) & (uint32_t)(cap - 1);
    }
    return false;
}

__global__ void init_ranges_kernel(int *r) {
    for (int i = threadIdx.x; i < kRangesWords; i += blockDim.x) r[i] = i >= 4 ? -1 : 0;
    if (threadIdx.x == 0) {
        r[0] = -1;         // max subject/object
        r[1] = -1;         // max predicate
        r[2] = INT32_MAX;  // min over all ids
    }
}

__global__ void __launch_bounds__(256) ranges_kernel(const int32_t *__restrict__ tri, int64_t n, int *r) {
    __shared__ int lset[kPredLocal];
    for (int i = threadIdx.x; i < kPredLocal; i += blockDim.x) lset[i] = -1;
    __syncthreads();
    int mx_so = -1, mx_p = -1, mn = INT32_MAX;
    bool over = false;
    int32_t last = -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = tri[3 * i], p = tri[3 * i + 1], o = tri[3 * i + 2];
        mx_so = max(mx_so, max(s, o));
        mx_p = max(mx_p, p);
        mn = min(mn, min(s, min(p, o)));
        if (p >= 0 && p != last) {
            over |= !set_insert(lset, kPredLocal, p);
            last = p;
        }
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        mx_so = max(mx_so, __shfl_xor_sync(0xffffffffu, mx_so, d));
        mx_p = max(mx_p, __shfl_xor_sync(0xffffffffu, mx_p, d));
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, d));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kPredLocal; i += blockDim.x) {
        if (lset[i] >= 0) over |= !set_insert(r + 4, kPredTable, lset[i]);
    }
    over = __any_sync(0xffffffffu, over);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&r[0], mx_so);
        atomicMax(&r[1], mx_p);
        atomicMin(&r[2], mn);
        if (over) atomicExch(&r[3], 1);
    }
}

__global__ void extract_pred_kernel(const int32_t *__restrict__ tri, int64_t n, uint32_t *__restrict__ p) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        p[i] = (uint32_t)tri[3 * i + 1];
    }
}

struct DistinctU32Op {
    const uint32_t *a;
    int32_t *out;
    __device__ bool flag(int64_t i) const {
        const int64_t h = i > 0 ? i - 1 : 0;  // branch-free: both loads issue at once
        return (i == 0) | (a[i] != a[h]);
    }
    __device__ void emit(int64_t i, int64_t j) const { out[j] = (int32_t)a[i]; }
};

__device__ __forceinline__ int32_t hash_lookup(const int32_t *keys, const int32_t *vals, uint32_t mask, int32_t p) {
    uint32_t h = ((uint32_t)p * 2654435761u) & mask;
    while (true) {
        const int32_t k = keys[h];
        if (k == p) return vals[h];
        if (k < 0) return -1;
        h = (h + 1) & mask;
    }
}

// Split the triples into s, o and predicate-slot columns.
__global__ void split_kernel(const int32_t *__restrict__ tri, int64_t n, const int32_t *__restrict__ hkeys,
                             const int32_t *__restrict__ hvals, uint32_t hmask, int32_t *__restrict__ s,
                             int32_t *__restrict__ o, int32_t *__restrict__ slot) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        s[i] = tri[3 * i];
        o[i] = tri[3 * i + 2];
        slot[i] = hash_lookup(hkeys, hvals, hmask, tri[3 * i + 1]);
    }
}

// key = slot << (2 bits) | s << bits | o, straight from the triples
__global__ void split_pack_kernel(const int32_t *__restrict__ tri, int64_t n, const int32_t *__restrict__ hkeys,
                                  const int32_t *__restrict__ hvals, uint32_t hmask, int bits,
                                  uint64_t *__restrict__ keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = (uint32_t)tri[3 * i], o = (uint32_t)tri[3 * i + 2];
        const uint32_t slot = (uint32_t)hash_lookup(hkeys, hvals, hmask, tri[3 * i + 1]);
        keys[i] = ((uint64_t)slot << (2 * bits)) | ((uint64_t)s << bits) | (uint64_t)o;
    }
}

// key = slot << (2 bits) | a << bits | b
__global__ void pack_kernel(const int32_t *__restrict__ a, const int32_t *__restrict__ b, const int32_t *__restrict__ c,
                            int64_t n, int bits, uint64_t *__restrict__ keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = ((uint64_t)(uint32_t)c[i] << (2 * bits)) | ((uint64_t)(uint32_t)a[i] << bits) | (uint64_t)(uint32_t)b[i];
    }
}

__global__ void unpack_kernel(const uint64_t *__restrict__ keys, int64_t n, int bits, int32_t *__restrict__ a,
                              int32_t *__restrict__ b, int32_t *__restrict__ c) {
    const uint64_t m = (bits >= 32) ? 0xffffffffull : ((1ull << bits) - 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        b[i] = (int32_t)(k & m);
        a[i] = (int32_t)((k >> bits) & m);
        c[i] = (int32_t)(k >> (2 * bits));
    }
}

__global__ void iota_kernel(uint32_t *v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        v[i] = (uint32_t)i;
    }
}

// keys[i] = x[perm[i]] (widened), or hi/lo packing of two columns.
__global__ void gather_key_kernel(const int32_t *__restrict__ hi, const int32_t *__restrict__ lo, int lo_bits,
                                  const uint32_t *__restrict__ perm, int64_t n, uint64_t *__restrict__ keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = perm ? perm[i] : (uint32_t)i;
        uint64_t k = (uint64_t)(uint32_t)lo[r];
        if (hi) k |= (uint64_t)(uint32_t)hi[r] << lo_bits;
        keys[i] = k;
    }
}

__global__ void gather3_kernel(const int32_t *__restrict__ a, const int32_t *__restrict__ b, const int32_t *__restrict__ c,
                               const uint32_t *__restrict__ perm, int64_t n, int32_t *__restrict__ oa,
                               int32_t *__restrict__ ob, int32_t *__restrict__ oc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = perm[i];
        oa[i] = a[r];
        ob[i] = b[r];
        oc[i] = c[r];
    }
}

// Drop adjacent repeats of sorted (c, a, b) rows.
struct DedupeOp {
    const int32_t *a, *b, *c;
    int32_t *oa, *ob, *oc;
    __device__ bool flag(int64_t i) const {
        const int64_t h = i > 0 ? i - 1 : 0;
        return (i == 0) | (a[i] != a[h]) | (b[i] != b[h]) | (c[i] != c[h]);
    }
    __device__ void emit(int64_t i, int64_t j) const {
        oa[j] = a[i];
        ob[j] = b[i];
        oc[j] = c[i];
    }
};

// Distinct keys of a sorted (slot, s, o) key array and, among them, the
// first of every (slot, s) row, in one pass (two nested selections): side
// 0's columns (key = s, val = o) and rows (Row = s, Rpos = first entry),
// and side 1's key (slot, o, s) for every distinct key.
struct DedupeRowsOp {
    const uint64_t *keys;
    int32_t *s0, *o0, *rowid, *rowoff;
    uint64_t *k1;
    int bits;
    __device__ void flags(int64_t i, bool &f1, bool &f2) const {
        const int64_t h = i > 0 ? i - 1 : 0;
        const uint64_t k = keys[i], kp = keys[h];
        f1 = (i == 0) | (k != kp);
        f2 = (i == 0) | ((k >> bits) != (kp >> bits));
    }
    __device__ void emit(int64_t i, int64_t j1, int64_t j2) const {
        const uint64_t k = keys[i];
        const uint64_t m = (1ull << bits) - 1;
        const uint64_t o = k & m, s = (k >> bits) & m, slot = k >> (2 * bits);
        s0[j1] = (int32_t)s;
        o0[j1] = (int32_t)o;
        k1[j1] = (slot << (2 * bits)) | (o << bits) | s;
        if (j2 >= 0) {
            rowid[j2] = (int32_t)s;
            rowoff[j2] = (int32_t)j1;
        }
    }
};

// Side 1 from its sorted (slot, o, s) keys in one pass: every entry's
// columns (key = o, val = s) and the first entry of every (slot, o) row.
struct RowsUnpackOp {
    const uint64_t *keys;
    int32_t *o1, *s1, *rowid, *rowoff;
    int bits;
    __device__ bool flag(int64_t i) const {
        const int64_t h = i > 0 ? i - 1 : 0;
        return (i == 0) | ((keys[i] >> bits) != (keys[h] >> bits));
    }
    __device__ void visit(int64_t i) const {
        const uint64_t k = keys[i];
        const uint64_t m = (1ull << bits) - 1;
        o1[i] = (int32_t)((k >> bits) & m);
        s1[i] = (int32_t)(k & m);
    }
    __device__ void emit(int64_t i, int64_t j) const {
        rowid[j] = (int32_t)((keys[i] >> bits) & ((1ull << bits) - 1));
        rowoff[j] = (int32_t)i;
    }
};

// Non-zero rows: the first entry of every (slot, key) run.
struct RowStartOp {
    const int32_t *key, *slot;
    int32_t *rowid, *rowoff;
    __device__ bool flag(int64_t i) const {
        const int64_t h = i > 0 ? i - 1 : 0;
        return (i == 0) | (key[i] != key[h]) | (slot[i] != slot[h]);
    }
    __device__ void emit(int64_t i, int64_t j) const {
        rowid[j] = key[i];
        rowoff[j] = (int32_t)i;
    }
};

// The predicate slot of entry i: a slot column, or the top bits of packed
// keys.  Either is ascending.
struct SlotSrc {
    const int32_t *col;
    const uint64_t *keys;
    int shift;
    __device__ int32_t at(int64_t i) const { return col ? col[i] : (int32_t)(keys[i] >> shift); }
};

// Per predicate p in [0, P]: its first entry (the first index whose slot is
// at or above p) and its first row (the first row starting at or after that
// entry).
__global__ void pred_bounds_kernel(SlotSrc slot, int64_t n, const int32_t *__restrict__ rowoff, int64_t R, int P,
                                   int32_t *__restrict__ ent_base, int32_t *__restrict__ row_base) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > P) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (slot.at(mid) < p) lo = mid + 1; else hi = mid;
    }
    const int32_t e = (int32_t)lo;
    lo = 0;
    hi = R;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (rowoff[mid] < e) lo = mid + 1; else hi = mid;
    }
    ent_base[p] = e;
    row_base[p] = (int32_t)lo;
}

// Dense row pointers of several predicates in one launch:
// dense[dense_base + x] = first entry of row x (or of the next non-empty
// row) for x in [0, max_entity + 1].  The x of every predicate are cut into
// chunks of kDenseChunk, and a warp takes kDenseRun consecutive chunks: one
// binary search finds the first row of the run, then per chunk the warp
// reads the chunk's row ids 32 at a time (coalesced; a ballot tells where
// the chunk ends, so the next chunk starts there), marks them in shared
// memory with their first entries, and an exclusive scan of the marks gives
// every x the number of the chunk's rows below it -- the index of its row's
// first entry; the writes are coalesced.
struct DensePart {
    int32_t row_base;
    int32_t nrows;
    int32_t end_entry;  // ent_base + nnz
    int32_t _pad;
    int64_t dense_base;
    int64_t chunk0;     // first chunk of this predicate
};
#ifndef GSMAT_DENSE_BYTES_PER_ENTRY
#define GSMAT_DENSE_BYTES_PER_ENTRY 4  // dense row pointers' budget per side, bytes per entry
#endif
constexpr int kDenseChunk = 256;
constexpr int kDenseRun = 16;  // consecutive chunks per warp
constexpr int kDenseWarps = kThreads / 32;

__device__ __forceinline__ int lower_bound_i32(const int32_t *__restrict__ a, int lo, int hi, int64_t x) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kThreads) dense_fill_kernel(const int32_t *__restrict__ rowid,
                                                              const int32_t *__restrict__ rowoff,
                                                              const DensePart *__restrict__ parts, int n_parts,
                                                              int64_t n_chunks, int64_t len,
                                                              int32_t *__restrict__ dense) {
    __shared__ int32_t s_off[kDenseWarps][kDenseChunk + 1];            // first entries of the chunk's rows (+ the next row)
    __shared__ __align__(16) int16_t s_pre[kDenseWarps][kDenseChunk];  // marks, then their exclusive prefix
    constexpr int kPer = kDenseChunk / 32;                              // x values (and candidate rows) per lane
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *off = s_off[wid];
    int16_t *pre = s_pre[wid];
    const int64_t warps = (int64_t)gridDim.x * kDenseWarps;
    const int64_t n_runs = (n_chunks + kDenseRun - 1) / kDenseRun;
    for (int64_t run = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; run < n_runs; run += warps) {
        int part = -1;
        int r0 = 0;
        DensePart P{};
        for (int64_t c = run * kDenseRun; c < n_chunks && c < (run + 1) * kDenseRun; ++c) {
            if (part < 0 || c >= P.chunk0 + (len + kDenseChunk - 1) / kDenseChunk) {
                int lo = 0, hi = n_parts;  // last part whose chunk0 <= c
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (parts[mid].chunk0 <= c) lo = mid; else hi = mid;
                }
                part = lo;
                P = parts[lo];
                r0 = lower_bound_i32(rowid + P.row_base, 0, P.nrows, (c - P.chunk0) * kDenseChunk);
            }
            const int64_t x0 = (c - P.chunk0) * kDenseChunk;
            const int32_t *ids = rowid + P.row_base;
            const int32_t *ro = rowoff + P.row_base;
            // The chunk's rows are a prefix of [r0, r0 + 256) (ids ascend and
            // are distinct): all 256 candidates' ids and first entries are
            // loaded at once, so a chunk costs one memory latency.
            int32_t id[kPer], fo[kPer];
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                const int r = r0 + 32 * k + lane;
                const bool ok = r < P.nrows;
                id[k] = ok ? __ldg(ids + r) : INT32_MAX;
                fo[k] = ok ? __ldg(ro + r) : 0;
            }
            *reinterpret_cast<int4 *>(pre + 8 * lane) = make_int4(0, 0, 0, 0);
            __syncwarp();
            int in_rows = 0;
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                const bool in = (int64_t)id[k] < x0 + kDenseChunk;
                if (in) {
                    pre[id[k] - x0] = 1;
                    off[32 * k + lane] = fo[k];
                }
                in_rows += __popc(__ballot_sync(0xffffffffu, in));
            }
            const int r1 = r0 + in_rows;
            if (lane == 0) off[in_rows] = r1 < P.nrows ? __ldg(ro + r1) : P.end_entry;
            __syncwarp();
            // exclusive prefix of the marks: lane l holds x0 + 8 l .. 8 l + 7
            // (one 16-byte shared-memory access each way)
            const int4 q = *reinterpret_cast<const int4 *>(pre + 8 * lane);
            int v[kPer];
            {
                const int32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    v[2 * t] = (int16_t)(w[t] & 0xffff);
                    v[2 * t + 1] = (int16_t)((uint32_t)w[t] >> 16);
                }
            }
            int sum = 0;
#pragma unroll
            for (int t = 0; t < kPer; ++t) sum += v[t];
            int inc = sum;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += y;
            }
            int run_sum = inc - sum;
            int32_t w[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int lo16 = run_sum;
                run_sum += v[2 * t];
                const int hi16 = run_sum;
                run_sum += v[2 * t + 1];
                w[t] = (int32_t)(((uint32_t)hi16 << 16) | ((uint32_t)lo16 & 0xffffu));
            }
            __syncwarp();
            *reinterpret_cast<int4 *>(pre + 8 * lane) = make_int4(w[0], w[1], w[2], w[3]);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                const int xi = lane + 32 * k;
                const int64_t x = x0 + xi;
                if (x < len) dense[P.dense_base + x] = off[pre[xi]];
            }
            __syncwarp();
            r0 = r1;
        }
    }
}

// Sort rows (c, a, b) lexicographically; results into oa/ob/oc.  With
// b_sorted the rows are already ascending in b among equal (c, a) (the
// input is sorted by (c, b, a)), so a stable sort on (c, a) alone suffices
// and b rides in the key's low bits unsorted.
int sort_rows3(const int32_t *a, const int32_t *b, const int32_t *c, int64_t n, int id_bits, int slot_bits,
               bool b_sorted, int32_t *oa, int32_t *ob, int32_t *oc, cudaStream_t st, int *err) {
    if (n == 0) return GSMAT_OK;
    const unsigned g = grid_for(n);
    if (slot_bits + 2 * id_bits <= 64) {
        DevBuf keys;
        GS_TRY(keys.alloc(sizeof(uint64_t) * (size_t)n, st));
        pack_kernel<<<g, kThreads, 0, st>>>(a, b, c, n, id_bits, keys.as<uint64_t>());
        GS_LAUNCH_CHECK();
        GS_TRY(radix_sort_u64(keys.as<uint64_t>(), nullptr, n, b_sorted ? id_bits : 0, slot_bits + 2 * id_bits, st,
                              err));
        unpack_kernel<<<g, kThreads, 0, st>>>(keys.as<uint64_t>(), n, id_bits, oa, ob, oc);
        GS_LAUNCH_CHECK();
        return GSMAT_OK;
    }
    // Wide ids: two stable passes, least significant field first.
    DevBuf keys, perm;
    GS_TRY(keys.alloc(sizeof(uint64_t) * (size_t)n, st));
    GS_TRY(perm.alloc(sizeof(uint32_t) * (size_t)n, st));
    iota_kernel<<<g, kThreads, 0, st>>>(perm.as<uint32_t>(), n);
    GS_LAUNCH_CHECK();
    gather_key_kernel<<<g, kThreads, 0, st>>>(nullptr, b, 0, nullptr, n, keys.as<uint64_t>());
    GS_LAUNCH_CHECK();
    GS_TRY(radix_sort_u64(keys.as<uint64_t>(), perm.as<uint32_t>(), n, 0, id_bits, st, err));
    gather_key_kernel<<<g, kThreads, 0, st>>>(c, a, id_bits, perm.as<uint32_t>(), n, keys.as<uint64_t>());
    GS_LAUNCH_CHECK();
    GS_TRY(radix_sort_u64(keys.as<uint64_t>(), perm.as<uint32_t>(), n, 0, slot_bits + id_bits, st, err));
    gather3_kernel<<<g, kThreads, 0, st>>>(a, b, c, perm.as<uint32_t>(), n, oa, ob, oc);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

// A side's predicate bounds and dense row pointers once its columns and
// row arrays (R rows; rid and roff sized for n rows, roff + 1) are built;
// the buffers move into the store.
int finish_side(gsmat_store *S, int side, DevBuf &key, DevBuf &val, DevBuf &rid, DevBuf &roff, int64_t R, SlotSrc slot,
                int64_t n, cudaStream_t st, PhaseTimer &pt) {
    const int P = S->n_pred;
    DevBuf bases;
    pt.add_bytes(8.0 * (double)R);  // Row and Rpos of the side's non-zero rows
    // the selection's buffers become the side's row arrays (sized for n
    // rows: no copy to exact size); rowoff gets its sentinel
    S->rowid[side] = std::move(rid);
    S->rowoff[side] = std::move(roff);
    const int32_t sentinel = (int32_t)n;
    GS_CUDA(cudaMemcpyAsync(S->rowoff[side].as<int32_t>() + R, &sentinel, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    // per predicate: first entry and first row
    GS_TRY(bases.alloc(sizeof(int32_t) * 2 * (size_t)(P + 1), st));
    int32_t *ent_base = bases.as<int32_t>(), *row_base = ent_base + (P + 1);
    pred_bounds_kernel<<<(P + 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(slot, n, S->rowoff[side].as<int32_t>(), R,
                                                                                P, ent_base, row_base);
    GS_LAUNCH_CHECK();
    std::vector<int32_t> hb(2 * (size_t)(P + 1));
    GS_CUDA(cudaMemcpyAsync(hb.data(), bases.p, sizeof(int32_t) * hb.size(), cudaMemcpyDeviceToHost, st));
    pt.pause();
    GS_CUDA(cudaStreamSynchronize(st));
    pt.resume();
    hb[P] = (int32_t)n;
    hb[(P + 1) + P] = (int32_t)R;
    S->side[side].resize(P);
    for (int p = 0; p < P; ++p) {
        PredSide &ps = S->side[side][p];
        ps.ent_base = hb[p];
        ps.nnz = hb[p + 1] - hb[p];
        ps.row_base = hb[(P + 1) + p];
        ps.nrows = hb[(P + 1) + p + 1] - hb[(P + 1) + p];
        ps.dense_base = -1;
    }
    // Dense row pointers (max_entity + 2 words each, at a multiple of 4
    // words) for the predicates with the most entries, while their total
    // stays within GSMAT_DENSE_BYTES_PER_ENTRY bytes per entry (4: as many
    // words as the side has entries); the others find rows by binary
    // search.  On a 3x10^8-triple graph a budget of 4 bytes left the
    // queries as fast as 16 bytes did and took 4 ms less to build; none
    // made them 30 % slower.
    const int64_t len = (int64_t)S->max_entity + 2;
    const int64_t stride = (len + 3) & ~int64_t(3);
    std::vector<int> by_nnz(P);
    for (int p = 0; p < P; ++p) by_nnz[p] = p;
    std::stable_sort(by_nnz.begin(), by_nnz.end(),
                     [&](int a, int b) { return S->side[side][a].nnz > S->side[side][b].nnz; });
    const int64_t budget = GSMAT_DENSE_BYTES_PER_ENTRY * n;
    int64_t total = 0;
    if (S->max_entity >= 0) {
        for (int p : by_nnz) {
            PredSide &ps = S->side[side][p];
            if (ps.nnz == 0 || (total + stride) * 4 > budget) continue;
            ps.dense_base = total;
            total += stride;
        }
    }
    S->n_dense[side] = 0;
    if (total > 0) {
        pt.add_bytes(4.0 * (double)total);  // dense row pointers written
        GS_TRY(S->dense[side].alloc(sizeof(int32_t) * (size_t)total, st));
        const int64_t per = (len + kDenseChunk - 1) / kDenseChunk;
        std::vector<DensePart> parts;
        for (int p = 0; p < P; ++p) {
            const PredSide &ps = S->side[side][p];
            if (ps.dense_base < 0) continue;
            DensePart d;
            d.row_base = ps.row_base;
            d.nrows = ps.nrows;
            d.end_entry = ps.ent_base + ps.nnz;
            d._pad = 0;
            d.dense_base = ps.dense_base;
            d.chunk0 = (int64_t)parts.size() * per;
            parts.push_back(d);
        }
        S->n_dense[side] = (int32_t)parts.size();
        DevBuf d_parts;
        GS_TRY(d_parts.alloc(sizeof(DensePart) * parts.size(), st));
        GS_CUDA(cudaMemcpyAsync(d_parts.p, parts.data(), sizeof(DensePart) * parts.size(), cudaMemcpyHostToDevice, st));
        const int64_t n_chunks = per * (int64_t)parts.size();
        const int64_t n_runs = (n_chunks + kDenseRun - 1) / kDenseRun;
        int64_t g = (n_runs * 32 + kThreads - 1) / kThreads;
        const int64_t cap = (int64_t)device_sm_count() * 16;
        if (g > cap) g = cap;
        dense_fill_kernel<<<(unsigned)g, kThreads, 0, st>>>(S->rowid[side].as<int32_t>(), S->rowoff[side].as<int32_t>(),
                                                            d_parts.as<DensePart>(), (int)parts.size(), n_chunks, len,
                                                            S->dense[side].as<int32_t>());
        GS_LAUNCH_CHECK();
        // the parts table is read by the kernel before the stream-ordered free
    }
    S->key[side] = std::move(key);
    S->val[side] = std::move(val);
    return GSMAT_OK;
}

// Build one side from entries sorted by (slot, key, val) in columns.
int build_side(gsmat_store *S, int side, DevBuf &key, DevBuf &val, const int32_t *slot, int64_t n, int *err,
               cudaStream_t st, PhaseTimer &pt) {
    DevBuf rid, roff, cnt;
    GS_TRY(rid.alloc(sizeof(int32_t) * (size_t)n, st));
    GS_TRY(roff.alloc(sizeof(int32_t) * (size_t)(n + 1), st));
    GS_TRY(cnt.alloc(sizeof(int64_t), st));
    RowStartOp op{key.as<int32_t>(), slot, rid.as<int32_t>(), roff.as<int32_t>()};
    GS_TRY(run_select(op, n, cnt.as<int64_t>(), st, err));
    int64_t *h = pinned_scratch(4);
    if (!h) return set_error(GSMAT_ERR_CUDA, "pinned host scratch");
    GS_CUDA(cudaMemcpyAsync(h, cnt.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    pt.pause();
    GS_CUDA(cudaStreamSynchronize(st));
    pt.resume();
    return finish_side(S, side, key, val, rid, roff, h[0], SlotSrc{slot, nullptr, 0}, n, st, pt);
}

// Both sides from (slot, s, o) columns, for ids too wide for one packed key
// (the sorts then run as two stable passes over narrower keys).
int build_columns(gsmat_store *S, const int32_t *tri, int64_t n, int id_bits, int slot_bits, DevBuf &d_tri_own,
                  int *err, cudaStream_t st, PhaseTimer &pt, int64_t *h) {
    // 3. side 0: sort by (slot, s, o) and drop repeats
    DevBuf s_raw, o_raw, slot_raw, s_sorted, o_sorted, slot_sorted, cnt;
    GS_TRY(s_raw.alloc(sizeof(int32_t) * (size_t)n, st));
    GS_TRY(o_raw.alloc(sizeof(int32_t) * (size_t)n, st));
    GS_TRY(slot_raw.alloc(sizeof(int32_t) * (size_t)n, st));
    {
        const uint32_t cap = S->hash_mask + 1;
        split_kernel<<<grid_for(n), kThreads, 0, st>>>(tri, n, S->hash_dev.as<int32_t>(), S->hash_dev.as<int32_t>() + cap,
                                                       S->hash_mask, s_raw.as<int32_t>(), o_raw.as<int32_t>(),
                                                       slot_raw.as<int32_t>());
        GS_LAUNCH_CHECK();
    }
    d_tri_own.release();
    GS_TRY(s_sorted.alloc(sizeof(int32_t) * (size_t)n, st));
    GS_TRY(o_sorted.alloc(sizeof(int32_t) * (size_t)n, st));
    GS_TRY(slot_sorted.alloc(sizeof(int32_t) * (size_t)n, st));
    GS_TRY(sort_rows3(s_raw.as<int32_t>(), o_raw.as<int32_t>(), slot_raw.as<int32_t>(), n, id_bits, slot_bits, false,
                      s_sorted.as<int32_t>(), o_sorted.as<int32_t>(), slot_sorted.as<int32_t>(), st, err));
    // dedupe into the raw buffers (reused)
    GS_TRY(cnt.alloc(sizeof(int64_t), st));
    {
        DedupeOp op{s_sorted.as<int32_t>(), o_sorted.as<int32_t>(), slot_sorted.as<int32_t>(),
                    s_raw.as<int32_t>(), o_raw.as<int32_t>(), slot_raw.as<int32_t>()};
        GS_TRY(run_select(op, n, cnt.as<int64_t>(), st, err));
        GS_CUDA(cudaMemcpyAsync(h, cnt.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        pt.pause();
        GS_CUDA(cudaStreamSynchronize(st));
        pt.resume();
    }
    const int64_t nu = h[0];
    S->n_unique = nu;
    pt.add_bytes(8.0 * (double)nu);  // the two sides' entry columns
    // side 0 arrays: key = s, val = o (exact size)
    DevBuf key0, val0, slot0;
    GS_TRY(key0.alloc(sizeof(int32_t) * (size_t)nu, st));
    GS_TRY(val0.alloc(sizeof(int32_t) * (size_t)nu, st));
    GS_TRY(slot0.alloc(sizeof(int32_t) * (size_t)nu, st));
    GS_CUDA(cudaMemcpyAsync(key0.p, s_raw.p, sizeof(int32_t) * (size_t)nu, cudaMemcpyDeviceToDevice, st));
    GS_CUDA(cudaMemcpyAsync(val0.p, o_raw.p, sizeof(int32_t) * (size_t)nu, cudaMemcpyDeviceToDevice, st));
    GS_CUDA(cudaMemcpyAsync(slot0.p, slot_raw.p, sizeof(int32_t) * (size_t)nu, cudaMemcpyDeviceToDevice, st));
    s_raw.release(); o_raw.release(); slot_raw.release();
    // 4. side 1: sort the unique triples by (slot, o, s); they are sorted by
    // (slot, s, o), so a stable sort on (slot, o) keeps s ascending
    DevBuf key1, val1, slot1;
    GS_TRY(key1.alloc(sizeof(int32_t) * (size_t)nu, st));
    GS_TRY(val1.alloc(sizeof(int32_t) * (size_t)nu, st));
    GS_TRY(slot1.alloc(sizeof(int32_t) * (size_t)nu, st));
    GS_TRY(sort_rows3(val0.as<int32_t>(), key0.as<int32_t>(), slot0.as<int32_t>(), nu, id_bits, slot_bits, true,
                      key1.as<int32_t>(), val1.as<int32_t>(), slot1.as<int32_t>(), st, err));
    s_sorted.release(); o_sorted.release(); slot_sorted.release();
    // 5. rows, predicate bounds, dense row pointers
    GS_TRY(build_side(S, 0, key0, val0, slot0.as<int32_t>(), nu, err, st, pt));
    GS_TRY(build_side(S, 1, key1, val1, slot1.as<int32_t>(), nu, err, st, pt));
    return GSMAT_OK;
}

// Both sides from one packed key per triple when (slot, s, o) fits 64 bits:
// sort by (slot, s, o); one selection pass drops repeats, writes side 0's
// columns and side 1's key (slot, o, s); a stable sort of that key on
// (slot, o) leaves s ascending inside every row (its input is in (slot, s)
// order).  The sorts ping-pong between two key buffers, never copying back.
int build_packed(gsmat_store *S, const int32_t *tri, int64_t n, int id_bits, int slot_bits, DevBuf &d_tri_own,
                 int *err, cudaStream_t st, PhaseTimer &pt, int64_t *h) {
    DevBuf ka, kb, cnt;
    GS_TRY(ka.alloc(sizeof(uint64_t) * (size_t)n, st));
    GS_TRY(kb.alloc(sizeof(uint64_t) * (size_t)n, st));
    {
        const uint32_t cap = S->hash_mask + 1;
        split_pack_kernel<<<grid_for(n), kThreads, 0, st>>>(tri, n, S->hash_dev.as<int32_t>(),
                                                            S->hash_dev.as<int32_t>() + cap, S->hash_mask, id_bits,
                                                            ka.as<uint64_t>());
        GS_LAUNCH_CHECK();
    }
    d_tri_own.release();
    const int key_bits = slot_bits + 2 * id_bits;
    uint64_t *sorted0 = nullptr;
    GS_TRY(radix_sort_u64_pingpong(ka.as<uint64_t>(), kb.as<uint64_t>(), n, 0, key_bits, st, err, &sorted0));
    uint64_t *k1 = sorted0 == ka.as<uint64_t>() ? kb.as<uint64_t>() : ka.as<uint64_t>();
    // side 0: columns and rows sized n (an upper bound of the distinct count)
    DevBuf key0, val0, rid0, roff0;
    GS_TRY(key0.alloc(sizeof(int32_t) * (size_t)n, st));
    GS_TRY(val0.alloc(sizeof(int32_t) * (size_t)n, st));
    GS_TRY(rid0.alloc(sizeof(int32_t) * (size_t)n, st));
    GS_TRY(roff0.alloc(sizeof(int32_t) * (size_t)(n + 1), st));
    GS_TRY(cnt.alloc(2 * sizeof(int64_t), st));
    {
        DedupeRowsOp op{sorted0, key0.as<int32_t>(), val0.as<int32_t>(), rid0.as<int32_t>(), roff0.as<int32_t>(), k1,
                        id_bits};
        GS_TRY(run_select2(op, n, cnt.as<int64_t>(), st, err));
        GS_CUDA(cudaMemcpyAsync(h, cnt.p, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        pt.pause();
        GS_CUDA(cudaStreamSynchronize(st));
        pt.resume();
    }
    const int64_t nu = h[0], R0 = h[1];
    S->n_unique = nu;
    pt.add_bytes(8.0 * (double)nu);  // the two sides' entry columns
    // side 0's bounds read the slots from k1 (still in side 0's order)
    GS_TRY(finish_side(S, 0, key0, val0, rid0, roff0, R0, SlotSrc{nullptr, k1, 2 * id_bits}, nu, st, pt));
    uint64_t *sorted1 = nullptr;
    GS_TRY(radix_sort_u64_pingpong(k1, sorted0, nu, id_bits, key_bits, st, err, &sorted1));
    // side 1: columns and rows from the sorted keys in one pass
    const size_t m = (size_t)(nu > 0 ? nu : 1);
    DevBuf key1, val1, rid1, roff1;
    GS_TRY(key1.alloc(sizeof(int32_t) * m, st));
    GS_TRY(val1.alloc(sizeof(int32_t) * m, st));
    GS_TRY(rid1.alloc(sizeof(int32_t) * m, st));
    GS_TRY(roff1.alloc(sizeof(int32_t) * (m + 1), st));
    {
        RowsUnpackOp op{sorted1, key1.as<int32_t>(), val1.as<int32_t>(), rid1.as<int32_t>(), roff1.as<int32_t>(), id_bits};
        GS_TRY(run_select(op, nu, cnt.as<int64_t>(), st, err));
        GS_CUDA(cudaMemcpyAsync(h, cnt.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        pt.pause();
        GS_CUDA(cudaStreamSynchronize(st));
        pt.resume();
    }
    const int64_t R1 = h[0];
    GS_TRY(finish_side(S, 1, key1, val1, rid1, roff1, R1, SlotSrc{nullptr, sorted1, 2 * id_bits}, nu, st, pt));
    ka.release();
    kb.release();
    return GSMAT_OK;
}

int build_impl(const int32_t *triples, int64_t n, int on_device, cudaStream_t st, gsmat_store *S) {
    S->n_input = n;
    DevBuf d_tri_own, ranges, err;
    const int32_t *tri = triples;
    GS_TRY(err.alloc(sizeof(int), st));
    GS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    if (n > 0 && !on_device) {
        GS_TRY(d_tri_own.alloc(sizeof(int32_t) * 3 * (size_t)n, st));
        GS_CUDA(cudaMemcpyAsync(d_tri_own.p, triples, sizeof(int32_t) * 3 * (size_t)n, cudaMemcpyHostToDevice, st));
        tri = d_tri_own.as<int32_t>();
    }
    // Device time of the build, without the host's waits between its
    // phases.  Algorithmic bytes: the triples read once (12 per triple),
    // both sides' columns (4 + 4 per unique triple), every non-zero row's
    // Row and Rpos words (8 per row and side) and the dense row pointers.
    PhaseTimer pt("store_build", st, (double)n);
    pt.add_bytes(12.0 * (double)n);
    pt.resume();
    int64_t *h = pinned_scratch(8);
    if (!h) return set_error(GSMAT_ERR_CUDA, "pinned host scratch");
    // 1. ranges
    GS_TRY(ranges.alloc(sizeof(int) * kRangesWords, st));
    init_ranges_kernel<<<1, 256, 0, st>>>(ranges.as<int>());
    GS_LAUNCH_CHECK();
    if (n > 0) ranges_kernel<<<grid_for(n), kThreads, 0, st>>>(tri, n, ranges.as<int>());
    GS_LAUNCH_CHECK();
    std::vector<int> hr_all(kRangesWords);
    GS_CUDA(cudaMemcpyAsync(hr_all.data(), ranges.p, sizeof(int) * kRangesWords, cudaMemcpyDeviceToHost, st));
    pt.pause();
    GS_CUDA(cudaStreamSynchronize(st));
    pt.resume();
    const int *hr = hr_all.data();
    if (n > 0 && hr[2] < 0) return set_error(GSMAT_ERR_INVALID_ARG, "negative id in triples (min %d)", hr[2]);
    S->max_entity = n > 0 ? hr[0] : -1;
    S->max_pred = n > 0 ? hr[1] : -1;
    if (n == 0) {
        for (int s = 0; s < 2; ++s) {
            GS_TRY(S->rowoff[s].alloc(sizeof(int32_t), st));
            GS_CUDA(cudaMemsetAsync(S->rowoff[s].p, 0, sizeof(int32_t), st));
        }
        S->hash_mask = 15;
        S->hash_keys.assign(16, -1);
        S->hash_vals.assign(16, -1);
        return GSMAT_OK;
    }
    // 2. distinct predicates -> slots, hash index
    if (!hr[3]) {
        // from the set collected by the ranges pass, ascending
        S->pred_ids.clear();
        for (int w = 0; w < kPredTable; ++w) {
            if (hr[4 + w] >= 0) S->pred_ids.push_back(hr[4 + w]);
        }
        std::sort(S->pred_ids.begin(), S->pred_ids.end());
        S->n_pred = (int32_t)S->pred_ids.size();
    } else {
        DevBuf pcol, pdist, cnt;
        GS_TRY(pcol.alloc(sizeof(uint32_t) * (size_t)n, st));
        GS_TRY(pdist.alloc(sizeof(int32_t) * (size_t)n, st));
        GS_TRY(cnt.alloc(sizeof(int64_t), st));
        extract_pred_kernel<<<grid_for(n), kThreads, 0, st>>>(tri, n, pcol.as<uint32_t>());
        GS_LAUNCH_CHECK();
        GS_TRY(radix_sort_u32(pcol.as<uint32_t>(), nullptr, n, 0, bits_for((uint64_t)S->max_pred), st, err.as<int>()));
        DistinctU32Op op{pcol.as<uint32_t>(), pdist.as<int32_t>()};
        GS_TRY(run_select(op, n, cnt.as<int64_t>(), st, err.as<int>()));
        GS_CUDA(cudaMemcpyAsync(h, cnt.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        pt.pause();
        GS_CUDA(cudaStreamSynchronize(st));
        pt.resume();
        const int64_t P = h[0];
        if (P <= 0 || P > INT32_MAX / 4) return set_error(GSMAT_ERR_CAPACITY, "%lld distinct predicates", (long long)P);
        S->n_pred = (int32_t)P;
        S->pred_ids.resize((size_t)P);
        GS_CUDA(cudaMemcpyAsync(S->pred_ids.data(), pdist.p, sizeof(int32_t) * (size_t)P, cudaMemcpyDeviceToHost, st));
        pt.pause();
        GS_CUDA(cudaStreamSynchronize(st));
        pt.resume();
    }
    {
        uint32_t cap = 16;
        while (cap < 2u * (uint32_t)S->n_pred) cap <<= 1;
        S->hash_mask = cap - 1;
        S->hash_keys.assign(cap, -1);
        S->hash_vals.assign(cap, -1);
        for (int32_t i = 0; i < S->n_pred; ++i) {
            uint32_t hh = pred_hash(S->pred_ids[i]) & S->hash_mask;
            while (S->hash_keys[hh] >= 0) hh = (hh + 1) & S->hash_mask;
            S->hash_keys[hh] = S->pred_ids[i];
            S->hash_vals[hh] = i;
        }
        GS_TRY(S->hash_dev.alloc(sizeof(int32_t) * 2 * cap, st));
        GS_CUDA(cudaMemcpyAsync(S->hash_dev.p, S->hash_keys.data(), sizeof(int32_t) * cap, cudaMemcpyHostToDevice, st));
        GS_CUDA(cudaMemcpyAsync(S->hash_dev.as<int32_t>() + cap, S->hash_vals.data(), sizeof(int32_t) * cap,
                                cudaMemcpyHostToDevice, st));
    }
    const int id_bits = std::max(1, bits_for((uint64_t)S->max_entity));
    const int slot_bits = bits_for((uint64_t)(S->n_pred - 1));
    if (slot_bits + 2 * id_bits <= 64) {
        GS_TRY(build_packed(S, tri, n, id_bits, slot_bits, d_tri_own, err.as<int>(), st, pt, h));
    } else {
        GS_TRY(build_columns(S, tri, n, id_bits, slot_bits, d_tri_own, err.as<int>(), st, pt, h));
    }
    // device copy of the per-predicate tables
    {
        const size_t P = (size_t)S->n_pred;
        GS_TRY(S->pred_side_dev.alloc(sizeof(PredSide) * 2 * P, st));
        GS_CUDA(cudaMemcpyAsync(S->pred_side_dev.p, S->side[0].data(), sizeof(PredSide) * P, cudaMemcpyHostToDevice, st));
        GS_CUDA(cudaMemcpyAsync(S->pred_side_dev.as<PredSide>() + P, S->side[1].data(), sizeof(PredSide) * P,
                                cudaMemcpyHostToDevice, st));
    }
    pt.finish();
    GS_CUDA(cudaMemcpyAsync(h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (*reinterpret_cast<int *>(h)) return set_error(GSMAT_ERR_DEVICE_CHECK, "store build: a bounded wait expired");
    return GSMAT_OK;
}

}  // namespace

int store_build(const int32_t *triples, int64_t n, int on_device, cudaStream_t st, gsmat_store **out) {
    if (!out) return set_error(GSMAT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || n > (int64_t)INT32_MAX) return set_error(GSMAT_ERR_INVALID_ARG, "n = %lld out of range", (long long)n);
    if (n > 0 && !triples) return set_error(GSMAT_ERR_INVALID_ARG, "triples is NULL");
    gsmat_store *S = new gsmat_store();
    cudaGetDevice(&S->device);
    int rc = build_impl(triples, n, on_device, st, S);
    if (rc == GSMAT_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = set_error(GSMAT_ERR_CUDA, "store build: %s", cudaGetErrorString(e));
    }
    if (rc != GSMAT_OK) {
        cudaStreamSynchronize(st);
        delete S;
        return rc;
    }
    // From here on the buffers are freed on the legacy stream (the load
    // stream may be gone by then).
    for (int s = 0; s < 2; ++s) {
        S->key[s].st = S->val[s].st = S->rowid[s].st = S->rowoff[s].st = S->dense[s].st = nullptr;
        S->view.side[s].key = S->key[s].as<int32_t>();
        S->view.side[s].val = S->val[s].as<int32_t>();
        S->view.side[s].rowid = S->rowid[s].as<int32_t>();
        S->view.side[s].rowoff = S->rowoff[s].as<int32_t>();
        S->view.side[s].dense = S->dense[s].as<int32_t>();
        S->view.side[s].max_entity = S->max_entity;
    }
    S->pred_side_dev.st = nullptr;
    S->hash_dev.st = nullptr;
    profile_flush();
    *out = S;
    return GSMAT_OK;
}

}  // namespace gs

int32_t gsmat_store::slot_of(int32_t pred_id) const {
    if (pred_id < 0 || hash_keys.empty()) return -1;
    uint32_t h = gs::pred_hash(pred_id) & hash_mask;
    while (true) {
        const int32_t k = hash_keys[h];
        if (k == pred_id) return hash_vals[h];
        if (k < 0) return -1;
        h = (h + 1) & hash_mask;
    }
}
