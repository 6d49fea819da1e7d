// Shared internals of libgsmat: status handling, the allocator hook, event
// timing, the device view of the SM store and the tile primitives (block
// scans and decoupled look-back) that the scan, compaction and join kernels
// build on.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/gsmat.h"

namespace gs {

// ---------------------------------------------------------------------------
// status

int set_error(int status, const char *fmt, ...);  // records detail, returns status
void clear_error();

#define GS_CUDA(call)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            return ::gs::set_error(GSMAT_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,    \
                                   cudaGetErrorString(e_));                                      \
        }                                                                                        \
    } while (0)

#define GS_TRY(expr)            \
    do {                        \
        int s_ = (expr);        \
        if (s_ != GSMAT_OK) {   \
            return s_;          \
        }                       \
    } while (0)

// After every kernel launch: counts it (gsmat_launch_count) and checks it.
void note_launch();
#define GS_LAUNCH_CHECK()      \
    do {                       \
        note_launch();         \
        GS_CUDA(cudaGetLastError()); \
    } while (0)

// ---------------------------------------------------------------------------
// device memory through the allocator hook

void *dev_alloc_raw(size_t bytes, cudaStream_t st);
void dev_free_raw(void *p, cudaStream_t st);

// Owning device buffer, freed in stream order on the stream it was made on.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), st(o.st) { o.p = nullptr; o.bytes = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; bytes = o.bytes; st = o.st;
            o.p = nullptr; o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    int alloc(size_t b, cudaStream_t s) {
        release();
        st = s;
        bytes = b;
        if (b == 0) return GSMAT_OK;
        p = dev_alloc_raw(b, s);
        if (!p) {
            bytes = 0;
            return set_error(GSMAT_ERR_OOM, "device allocation of %zu bytes failed", b);
        }
        return GSMAT_OK;
    }
    void release() {
        if (p) dev_free_raw(p, st);
        p = nullptr;
        bytes = 0;
    }
    template <class T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// per-launch event timing (enabled by gsmat_profile_enable)

bool profile_on();
// A timed region on a stream; no-op when profiling is off.
struct KernelTimer {
    const char *name;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    double bytes, items;
    bool counts;
    // counts_call = false: a further segment of a call already counted (its
    // time and bytes add to the family, its call count does not)
    KernelTimer(const char *n, cudaStream_t s, double algo_bytes, double n_items, bool counts_call = true);
    void stop();
    ~KernelTimer() { if (a) stop(); }
};

// The device time of one call made of several stream segments (the host
// waits between them): segments are timed separately and add up to one
// call of the family, so host round trips are not counted as device time.
struct PhaseTimer {
    const char *name;
    cudaStream_t st;
    double bytes = 0, items = 0;
    bool started = false;
    KernelTimer *cur = nullptr;
    PhaseTimer(const char *n, cudaStream_t s, double n_items) : name(n), st(s), items(n_items) {}
    PhaseTimer(const PhaseTimer &) = delete;
    PhaseTimer &operator=(const PhaseTimer &) = delete;
    void resume() {
        if (cur) return;
        cur = new KernelTimer(name, st, 0.0, started ? 0.0 : items, !started);
        started = true;
    }
    void pause() {
        if (!cur) return;
        cur->stop();
        delete cur;
        cur = nullptr;
    }
    // algorithmic bytes, attributed to the segment in progress (or the next)
    void add_bytes(double b) { bytes += b; }
    void finish() {
        resume();
        cur->bytes = bytes;
        pause();
    }
    ~PhaseTimer() { pause(); }
};
// Resolve finished timers of the calling thread into the global counters
// (call after the stream they were recorded on has been synchronised).
void profile_flush();

// ---------------------------------------------------------------------------
// pinned host scratch for small device->host reads (one per host thread)

int64_t *pinned_scratch(int n_words);
// Device alias of a pointer into the calling thread's pinned scratch (null
// outside it).
void *pinned_scratch_device(const void *host_ptr);
// h_dst[0..n) = the 8-byte words at d_src, written by a one-warp kernel on
// `st` into the mapped scratch (h_dst[0..n] must lie in it: h_dst[n] takes a
// completion tag); returns once `st` has reached the copy.
int read_words(const void *d_src, int64_t *h_dst, int n_words, cudaStream_t st);
// Returns once `st` has finished its work so far (as cudaStreamSynchronize,
// woken by a completion tag the stream writes into the mapped scratch's word
// kScratchTagWord, which no other use of the scratch touches).
constexpr int kScratchTagWord = 1023;
int wait_stream(cudaStream_t st);

// ---------------------------------------------------------------------------
// device view of the store

// One predicate on one side (side 0: rows by subject, CSR; side 1: rows by
// object, CSC).  Entry and row indices are global into the side's arrays.
struct PredSide {
    int32_t ent_base;   // first entry
    int32_t nnz;        // number of entries (m of Sec. 5.3)
    int32_t row_base;   // first non-zero row (auxiliary-array row)
    int32_t nrows;      // number of non-zero rows
    int64_t dense_base; // offset of a dense row pointer (max_entity + 2 words), or -1
};

// One side of the store (side 0: rows by subject; side 1: rows by object).
struct SideView {
    const int32_t *key;    // per entry: the row id (s on side 0, o on side 1)
    const int32_t *val;    // per entry: the other end
    const int32_t *rowid;  // per non-zero row: its id (Row of Sec. 6.3)
    const int32_t *rowoff; // per non-zero row: first entry; rowoff[R] = n (Rpos; Num = difference)
    const int32_t *dense;  // dense row pointers of the predicates that have one
    int32_t max_entity;
};

struct StoreView {
    SideView side[2];
};

// Entry range [first, last) of row x of predicate side ps; empty if absent.
__device__ __forceinline__ int2 row_range(const SideView &sv, const PredSide &ps, int32_t x) {
    if (ps.nnz == 0 || x < 0) return make_int2(0, 0);
    if (ps.dense_base >= 0) {
        if (x > sv.max_entity) return make_int2(0, 0);
        const int32_t *rp = sv.dense + ps.dense_base + x;
        return make_int2(__ldg(rp), __ldg(rp + 1));
    }
    const int32_t *ids = sv.rowid + ps.row_base;
    int lo = 0, hi = ps.nrows;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (__ldg(ids + mid) < x) lo = mid + 1; else hi = mid;
    }
    if (lo < ps.nrows && __ldg(ids + lo) == x) {
        const int32_t *ro = sv.rowoff + ps.row_base + lo;
        return make_int2(__ldg(ro), __ldg(ro + 1));
    }
    return make_int2(0, 0);
}

// row_range for N values at once, with every lookup's loads in flight
// together: the dense pointers' loads, or the binary searches advanced in
// lockstep (one independent load per value per step).  ok[j] false: r[j] =
// (0, 0).
template <int N>
__device__ __forceinline__ void row_ranges(const SideView &sv, const PredSide &ps, const int32_t (&x)[N],
                                           const bool (&ok)[N], int2 (&r)[N]) {
    if (ps.nnz == 0) {
#pragma unroll
        for (int j = 0; j < N; ++j) r[j] = make_int2(0, 0);
        return;
    }
    if (ps.dense_base >= 0) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const bool in = ok[j] && x[j] >= 0 && x[j] <= sv.max_entity;
            const int32_t *rp = sv.dense + ps.dense_base + (in ? x[j] : 0);
            r[j] = in ? make_int2(__ldg(rp), __ldg(rp + 1)) : make_int2(0, 0);
        }
        return;
    }
    const int32_t *ids = sv.rowid + ps.row_base;
    int lo[N], hi[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        lo[j] = 0;
        hi[j] = (ok[j] && x[j] >= 0) ? ps.nrows : 0;
    }
    for (int span = ps.nrows; span > 0; span >>= 1) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (lo[j] < hi[j]) {
                const int mid = (lo[j] + hi[j]) >> 1;
                if (__ldg(ids + mid) < x[j]) lo[j] = mid + 1; else hi[j] = mid;
            }
        }
    }
    int32_t at[N];
#pragma unroll
    for (int j = 0; j < N; ++j) at[j] = (ok[j] && x[j] >= 0 && lo[j] < ps.nrows) ? __ldg(ids + lo[j]) : -1;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int32_t *ro = sv.rowoff + ps.row_base + lo[j];
        r[j] = (at[j] == x[j] && at[j] >= 0) ? make_int2(__ldg(ro), __ldg(ro + 1)) : make_int2(0, 0);
    }
}

// Is v among the sorted entries val[first, last)?
__device__ __forceinline__ bool sorted_contains(const int32_t *__restrict__ vals, int first, int last, int32_t v) {
    int lo = first, hi = last;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (__ldg(vals + mid) < v) lo = mid + 1; else hi = mid;
    }
    return lo < last && __ldg(vals + lo) == v;
}

// ---------------------------------------------------------------------------
// warp / block scans

__device__ __forceinline__ int64_t warp_inclusive_sum(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__device__ __forceinline__ int64_t warp_sum(int64_t v) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Exclusive sum over the block of one value per thread, in thread order.
// smem: int64_t[BLOCK / 32 + 1].  Returns the thread's exclusive prefix and
// the block total in *total.  Contains __syncthreads.
template <int BLOCK>
__device__ __forceinline__ int64_t block_exclusive_sum(int64_t v, int64_t *smem, int64_t *total) {
    constexpr int W = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = warp_inclusive_sum(v);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < W ? smem[lane] : 0;
        int64_t wi = warp_inclusive_sum(w);
        if (lane < W) smem[lane] = wi - w;
        if (lane == W - 1) smem[W] = wi;
    }
    __syncthreads();
    int64_t ex = smem[warp] + inc - v;
    *total = smem[W];
    __syncthreads();
    return ex;
}

// ---------------------------------------------------------------------------
// decoupled look-back over tiles (single-pass prefix sums)

// Tile descriptor word: bits 62-63 = state, bits 0-61 = value (>= 0).
constexpr uint64_t kTileInvalid = 0;
constexpr uint64_t kTileAggregate = 1;
constexpr uint64_t kTilePrefix = 2;
constexpr uint64_t kValueMask = (uint64_t(1) << 62) - 1;
// A bounded wait: after this many polls (each followed by a short sleep)
// the kernel records an error and treats the missing predecessor as 0.
constexpr int kLookbackPollLimit = 1 << 22;

// Scratch of one single-pass launch: tile descriptors, the dynamic tile
// counter and an error word.  All must be zero before the launch.
struct LookbackScratch {
    unsigned long long *status; // [n_tiles]
    unsigned int *tile_counter; // [1]
    int *error;                 // [1]; set to 1 if a bounded wait expired
    int poll_limit;             // polls before a wait gives up (kLookbackPollLimit)
};

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}

// Obtain this CTA's tile id in launch order (guarantees that every smaller
// tile id belongs to a CTA that already started).  smem: one int.
__device__ __forceinline__ int acquire_tile_id(const LookbackScratch &ls, int *smem_tile) {
    if (threadIdx.x == 0) *smem_tile = (int)atomicAdd(ls.tile_counter, 1u);
    __syncthreads();
    int t = *smem_tile;
    __syncthreads();
    return t;
}

// Called by every thread of the CTA with the tile's aggregate (same value in
// all threads).  Returns the exclusive prefix of all earlier tiles.
// smem: one int64.  Warp 0 performs the look-back 32 predecessors at a time.
__device__ __forceinline__ int64_t tile_lookback(const LookbackScratch &ls, int tile, int64_t aggregate,
                                                 int64_t *smem_prefix) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        int64_t exclusive = 0;
        if (tile == 0) {
            if (lane == 0) {
                atomicExch(&ls.status[0], (unsigned long long)((kTilePrefix << 62) | ((uint64_t)aggregate & kValueMask)));
            }
        } else {
            if (lane == 0) {
                atomicExch(&ls.status[tile],
                           (unsigned long long)((kTileAggregate << 62) | ((uint64_t)aggregate & kValueMask)));
            }
            int base = tile - 1;
            bool failed = false;
            while (true) {
                const int j = base - lane;
                unsigned long long w;
                int polls = 0;
                while (true) {
                    w = (j >= 0) ? ld_volatile_u64(&ls.status[j]) : (unsigned long long)(kTilePrefix << 62);
                    const bool ready = (w >> 62) != kTileInvalid;
                    if (__all_sync(0xffffffffu, ready)) break;
                    if (++polls > ls.poll_limit) {
                        failed = true;
                        break;
                    }
                    __nanosleep(64);
                }
                if (failed) break;
                const unsigned prefix_mask = __ballot_sync(0xffffffffu, (w >> 62) == kTilePrefix);
                const int stop = prefix_mask ? (__ffs(prefix_mask) - 1) : 31;
                int64_t v = (lane <= stop) ? (int64_t)(w & kValueMask) : 0;
                exclusive += warp_sum(v);
                if (prefix_mask) break;
                base -= 32;
            }
            if (failed && lane == 0) atomicExch(ls.error, 1);
            if (lane == 0) {
                atomicExch(&ls.status[tile],
                           (unsigned long long)((kTilePrefix << 62) | ((uint64_t)(exclusive + aggregate) & kValueMask)));
            }
        }
        if (lane == 0) *smem_prefix = exclusive;
    }
    __syncthreads();
    int64_t r = *smem_prefix;
    __syncthreads();
    return r;
}

// Allocates and zeroes look-back scratch for n_tiles tiles.
struct LookbackBuf {
    DevBuf buf;
    LookbackScratch view{};
    // err_word (device int, may be null): where an expired wait is reported;
    // defaults to a word inside the scratch.
    int make(int64_t n_tiles, cudaStream_t st, int *err_word = nullptr) {
        size_t words = (size_t)(n_tiles > 0 ? n_tiles : 1);
        size_t bytes = words * 8 + 16;
        GS_TRY(buf.alloc(bytes, st));
        GS_CUDA(cudaMemsetAsync(buf.p, 0, bytes, st));
        view.status = buf.as<unsigned long long>();
        view.tile_counter = reinterpret_cast<unsigned int *>(buf.as<char>() + words * 8);
        view.error = err_word ? err_word : reinterpret_cast<int *>(buf.as<char>() + words * 8 + 4);
        view.poll_limit = kLookbackPollLimit;
        return GSMAT_OK;
    }
};

// ---------------------------------------------------------------------------
// internal entry points shared between translation units

// Stable radix sort on bits [begin_bit, end_bit); a bounded wait that
// expires sets *err_word (device int) when given.
int radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit, cudaStream_t st,
                   int *err_word = nullptr);
int radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit, cudaStream_t st,
                   int *err_word = nullptr);
// Keys only, with the caller's second buffer `alt` (n words): *sorted is
// set to whichever of keys / alt holds the sorted keys (no copy back).
int radix_sort_u64_pingpong(uint64_t *keys, uint64_t *alt, int64_t n, int begin_bit, int end_bit, cudaStream_t st,
                            int *err_word, uint64_t **sorted);
// As radix_sort_u64 with a 64-bit payload (required).
int radix_sort_u64_wide(uint64_t *keys, uint64_t *vals, int64_t n, int begin_bit, int end_bit, cudaStream_t st,
                        int *err_word = nullptr);
// Exclusive scan of int32 counts into int64[n+1]; *err_word (device int) is
// set if a bounded wait expired (may be null).
int exclusive_scan_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t st, int *err_word);
// The scan kernel over four tiles with tile 0 never handed out, so that the
// other tiles' look-back waits run out after poll_limit polls; returns
// GSMAT_ERR_DEVICE_CHECK when they did (the designed outcome).
int selftest_wait_expiry(int poll_limit, cudaStream_t st);

// exclusive_scan_i32 with its scratch in a static device array (no
// allocation); n at most exclusive_scan_i32_noalloc_max().
int exclusive_scan_i32_noalloc(const int32_t *in, int64_t *out, int64_t n, cudaStream_t st);
int64_t exclusive_scan_i32_noalloc_max();

// In-place exclusive scan of uint32 values whose total fits in 32 bits.
int exclusive_scan_u32_inplace(uint32_t *data, int64_t n, cudaStream_t st);

// Stable selection: out[j] = in[i] for the i with flags[i] != 0, in order;
// *d_count (device int64) receives the number selected.
int select_flagged_i32(const int32_t *in, const uint8_t *flags, int32_t *out, int64_t n, int64_t *d_count,
                       cudaStream_t st, int *err_word);

int device_sm_count();

// Grid for a grid-stride loop over n items: enough CTAs to cover n, capped
// at 16 per SM.
inline unsigned grid_1d(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

inline int bits_for(uint64_t max_value) {
    int b = 0;
    while (b < 64 && (max_value >> b) != 0) b++;
    return b;
}

}  // namespace gs
