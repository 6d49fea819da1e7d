// Stable LSD radix sort of 32/64-bit keys with an optional 32-bit payload.
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
#include "common.cuh"

namespace gs {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kBins = 256;
constexpr int kMaxPasses = 8;

template <class K>
struct SortTraits;
template <>
struct SortTraits<uint64_t> {
    static constexpr int kItems = 12;
};
template <>
struct SortTraits<uint32_t> {
    static constexpr int kItems = 16;
};

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

template <class K>
__global__ void __launch_bounds__(kBlock) onesweep_histogram(const K *__restrict__ keys, int64_t n, int begin_bit,
                                                            int end_bit, int n_pass, uint32_t *__restrict__ hist) {
    extern __shared__ uint32_t hsm[];  // [kWarps][n_pass][kBins]
    const int per_warp = n_pass * kBins;
    for (int i = threadIdx.x; i < kWarps * per_warp; i += kBlock) hsm[i] = 0;
    __syncthreads();
    uint32_t *wh = hsm + (threadIdx.x >> 5) * per_warp;
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
        const K k = __ldg(keys + i);
        for (int p = 0; p < n_pass; ++p) {
            const int shift = begin_bit + 8 * p;
            const int width = end_bit - shift < 8 ? end_bit - shift : 8;
            atomicAdd(&wh[p * kBins + digit_of(k, shift, (1 << width) - 1)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < per_warp; i += kBlock) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += hsm[w * per_warp + i];
        if (s) atomicAdd(hist + i, s);
    }
}

template <class K, bool HasVals>
__global__ void __launch_bounds__(kBlock, 4) onesweep_pass(const K *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                                                       K *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                                                       int64_t n, int shift, int mask,
                                                       const uint32_t *__restrict__ hist_pass,
                                                       unsigned long long *__restrict__ desc,
                                                       unsigned int *__restrict__ tile_counter, uint32_t epoch,
                                                       int *__restrict__ err) {
    constexpr int ITEMS = SortTraits<K>::kItems;
    constexpr int TILE = kBlock * ITEMS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *skeys = reinterpret_cast<K *>(smem_raw);
    uint32_t *svals = reinterpret_cast<uint32_t *>(skeys + TILE);
    uint32_t *whist = svals + (HasVals ? TILE : 0);  // [kWarps][kBins]
    uint32_t *tstart = whist + kWarps * kBins;
    uint32_t *gbase = tstart + kBins;
    __shared__ int64_t scan_tmp[kWarps + 1];
    __shared__ int tile_sm;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) tile_sm = (int)atomicAdd(tile_counter, 1u);
    for (int i = threadIdx.x; i < kWarps * kBins; i += kBlock) whist[i] = 0;
    __syncthreads();
    const int tile = tile_sm;
    const int64_t t0 = (int64_t)tile * TILE;
    const int valid = (int)((n - t0) < TILE ? (n - t0) : TILE);
    const unsigned lt_mask = (1u << lane) - 1u;
    uint32_t *wh = whist + warp * kBins;

    K k[ITEMS];
    uint32_t v[ITEMS];
    uint32_t dr[ITEMS];  // rank within the warp << 8 | digit
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        // warp-striped: stable order inside the tile is (warp, j, lane)
        const int idx = warp * (32 * ITEMS) + j * 32 + lane;
        if (idx < valid) {
            k[j] = keys_in[t0 + idx];
            v[j] = HasVals ? vals_in[t0 + idx] : 0u;
            dr[j] = (uint32_t)digit_of(k[j], shift, mask);
        } else {
            k[j] = ~K(0);
            v[j] = 0u;
            dr[j] = kBins - 1;  // padding ranks last in the last bucket
        }
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int d = (int)dr[j];
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader) {
            base = wh[d];
            wh[d] = base + (uint32_t)__popc(peers);
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        dr[j] = ((base + (uint32_t)__popc(peers & lt_mask)) << 8) | (uint32_t)d;
        __syncwarp();
    }
    __syncthreads();
    // per digit (thread d): cross-warp prefix, tile count, tile start
    const int d = threadIdx.x;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = whist[w * kBins + d];
        whist[w * kBins + d] = cnt;
        cnt += c;
    }
    int64_t tot;
    const int64_t ts = block_exclusive_sum<kBlock>((int64_t)cnt, scan_tmp, &tot);
    tstart[d] = (uint32_t)ts;
    const uint32_t real = cnt - (d == kBins - 1 ? (uint32_t)(TILE - valid) : 0u);
    // global start of digit d in this pass (exclusive scan of the histogram)
    const int64_t dbase = block_exclusive_sum<kBlock>((int64_t)__ldg(hist_pass + d), scan_tmp, &tot);
    // publish this tile's count of digit d, then look back for the earlier ones
    uint64_t excl = 0;
    if (tile == 0) {
        atomicExch(desc + d, desc_pack(epoch, kDescPrefix, real));
    } else {
        atomicExch(desc + (int64_t)tile * kBins + d, desc_pack(epoch, kDescAggregate, real));
        int j = tile - 1;
        int polls = 0;
        while (j >= 0) {
            const unsigned long long w = *(const volatile unsigned long long *)(desc + (int64_t)j * kBins + d);
            const uint64_t state = (w >> 54) & 3;
            if ((uint32_t)(w >> 56) != epoch || state == 0) {
                if (++polls > kLookbackPollLimit) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(32);
                continue;
            }
            excl += w & ((1ull << 54) - 1);
            if (state == kDescPrefix) break;
            --j;
        }
        atomicExch(desc + (int64_t)tile * kBins + d, desc_pack(epoch, kDescPrefix, excl + real));
    }
    gbase[d] = (uint32_t)(dbase + (int64_t)excl);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t dd = dr[j] & 0xffu;
        const uint32_t pos = tstart[dd] + wh[dd] + (dr[j] >> 8);
        skeys[pos] = k[j];
        if (HasVals) svals[pos] = v[j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < valid; i += kBlock) {
        const K kk = skeys[i];
        const int dd = digit_of(kk, shift, mask);
        const uint32_t dst = gbase[dd] + ((uint32_t)i - tstart[dd]);
        keys_out[dst] = kk;
        if (HasVals) vals_out[dst] = svals[i];
    }
}

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 148;
        }
        cached[dev] = v;
    }
    return cached[dev];
}

template <class K, bool HasVals>
int pass_smem_bytes() {
    constexpr int TILE = kBlock * SortTraits<K>::kItems;
    return TILE * (int)sizeof(K) + (HasVals ? TILE * 4 : 0) + (kWarps * kBins + 2 * kBins) * 4;
}

template <class K, bool HasVals>
int set_pass_attributes() {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!done[dev]) {
        GS_CUDA(cudaFuncSetAttribute(onesweep_pass<K, HasVals>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     pass_smem_bytes<K, HasVals>()));
        GS_CUDA(cudaFuncSetAttribute(onesweep_pass<K, HasVals>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared));
        GS_CUDA(cudaFuncSetAttribute(onesweep_histogram<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kWarps * kMaxPasses * kBins * 4));
        done[dev] = true;
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
    constexpr int TILE = kBlock * SortTraits<K>::kItems;
    const int64_t ntiles = (n + TILE - 1) / TILE;
    const int n_pass = (end_bit - begin_bit + 7) / 8;
    const int attr_rc = vals ? set_pass_attributes<K, true>() : set_pass_attributes<K, false>();
    if (attr_rc != GSMAT_OK) return attr_rc;

    // scratch: digit histograms | tile counters | error word | descriptors
    const size_t off_cnt = round_up(sizeof(uint32_t) * kBins * n_pass, 256);
    const size_t off_err = off_cnt + sizeof(uint32_t) * kMaxPasses;
    const size_t off_desc = round_up(off_err + sizeof(int), 256);
    const size_t meta_bytes = off_desc + sizeof(unsigned long long) * kBins * (size_t)ntiles;
    DevBuf alt_k, alt_v, meta;
    GS_TRY(alt_k.alloc(sizeof(K) * (size_t)n, st));
    if (vals) GS_TRY(alt_v.alloc(sizeof(uint32_t) * (size_t)n, st));
    GS_TRY(meta.alloc(meta_bytes, st));
    GS_CUDA(cudaMemsetAsync(meta.p, 0, meta_bytes, st));
    uint32_t *hist = meta.as<uint32_t>();
    unsigned int *counters = reinterpret_cast<unsigned int *>(meta.as<char>() + off_cnt);
    int *err = err_word ? err_word : reinterpret_cast<int *>(meta.as<char>() + off_err);
    unsigned long long *desc = reinterpret_cast<unsigned long long *>(meta.as<char>() + off_desc);

    KernelTimer t(timer_name, st, (double)n * (2.0 * sizeof(K) + (vals ? 8.0 : 0.0)) * n_pass, (double)n);
    {
        int64_t g = (n + kBlock * 16 - 1) / (kBlock * 16);
        const int64_t cap = (int64_t)sm_count() * 2;
        if (g > cap) g = cap;
        if (g < 1) g = 1;
        onesweep_histogram<K><<<(unsigned)g, kBlock, kWarps * n_pass * kBins * 4, st>>>(keys, n, begin_bit, end_bit,
                                                                                        n_pass, hist);
        GS_LAUNCH_CHECK();
    }
    K *src_k = keys, *dst_k = alt_k.as<K>();
    uint32_t *src_v = vals, *dst_v = alt_v.as<uint32_t>();
    for (int p = 0; p < n_pass; ++p) {
        const int shift = begin_bit + 8 * p;
        const int width = end_bit - shift < 8 ? end_bit - shift : 8;
        const int mask = (1 << width) - 1;
        if (vals) {
            onesweep_pass<K, true><<<(unsigned)ntiles, kBlock, pass_smem_bytes<K, true>(), st>>>(
                src_k, src_v, dst_k, dst_v, n, shift, mask, hist + p * kBins, desc, counters + p, (uint32_t)(p + 1), err);
        } else {
            onesweep_pass<K, false><<<(unsigned)ntiles, kBlock, pass_smem_bytes<K, false>(), st>>>(
                src_k, nullptr, dst_k, nullptr, n, shift, mask, hist + p * kBins, desc, counters + p, (uint32_t)(p + 1),
                err);
        }
        GS_LAUNCH_CHECK();
        K *tk = src_k; src_k = dst_k; dst_k = tk;
        uint32_t *tv = src_v; src_v = dst_v; dst_v = tv;
    }
    t.stop();
    if (src_k != keys) {
        GS_CUDA(cudaMemcpyAsync(keys, src_k, sizeof(K) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        if (vals) GS_CUDA(cudaMemcpyAsync(vals, src_v, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    }
    return GSMAT_OK;
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

int device_sm_count() { return sm_count(); }

}  // namespace gs
