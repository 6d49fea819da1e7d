// Stable LSD radix sort of 32/64-bit keys with an optional 32-bit payload.
//
// Used by the store builder (sorting the triple set by (p, s, o) and
// (p, o, s), which lays out every predicate's matrix M_h of Sec. 5.3 row by
// row) and by the final canonical ordering of a result table.
//
// Per 8-bit digit pass, three kernels over an even share of the input per
// CTA: an upsweep digit histogram per CTA, one scan of the digit-major
// histogram table, and a downsweep that ranks each tile of keys stably
// (warp match_any over the digit, per-warp counters, cross-warp prefix),
// stages the tile in shared memory in digit order and writes each digit's
// run to its global offset, so that the writes of a run are contiguous.
#include "common.cuh"

namespace gs {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kBins = 256;

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

template <class K>
__global__ void __launch_bounds__(kBlock) radix_upsweep(const K *__restrict__ keys, int64_t n, int64_t span,
                                                       int shift, int mask, int num_ctas,
                                                       uint32_t *__restrict__ counts) {
    __shared__ uint32_t hist[kWarps * kBins];
    for (int i = threadIdx.x; i < kWarps * kBins; i += kBlock) hist[i] = 0;
    __syncthreads();
    const int64_t begin = (int64_t)blockIdx.x * span;
    const int64_t end = begin + span < n ? begin + span : n;
    uint32_t *wh = hist + (threadIdx.x >> 5) * kBins;
    int64_t i = begin + threadIdx.x;
    for (; i + 3 * kBlock < end; i += 4 * kBlock) {
        K a = __ldg(keys + i), b = __ldg(keys + i + kBlock), c = __ldg(keys + i + 2 * kBlock),
          d = __ldg(keys + i + 3 * kBlock);
        atomicAdd(&wh[digit_of(a, shift, mask)], 1u);
        atomicAdd(&wh[digit_of(b, shift, mask)], 1u);
        atomicAdd(&wh[digit_of(c, shift, mask)], 1u);
        atomicAdd(&wh[digit_of(d, shift, mask)], 1u);
    }
    for (; i < end; i += kBlock) atomicAdd(&wh[digit_of(__ldg(keys + i), shift, mask)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += kBlock) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += hist[w * kBins + d];
        counts[(int64_t)d * num_ctas + blockIdx.x] = s;
    }
}

template <class K, bool HasVals>
__global__ void __launch_bounds__(kBlock) radix_downsweep(const K *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                                                         K *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                                                         int64_t n, int64_t span, int shift, int mask, int num_ctas,
                                                         const uint32_t *__restrict__ offsets) {
    constexpr int ITEMS = SortTraits<K>::kItems;
    constexpr int TILE = kBlock * ITEMS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *skeys = reinterpret_cast<K *>(smem_raw);
    uint32_t *svals = reinterpret_cast<uint32_t *>(skeys + TILE);
    uint32_t *whist = svals + (HasVals ? TILE : 0);
    uint32_t *running = whist + kWarps * kBins;
    uint32_t *tstart = running + kBins;
    uint32_t *tcount = tstart + kBins;
    __shared__ int64_t scan_tmp[kWarps + 1];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kBins; d += kBlock) running[d] = offsets[(int64_t)d * num_ctas + blockIdx.x];
    const int64_t begin = (int64_t)blockIdx.x * span;
    const int64_t end = begin + span < n ? begin + span : n;
    const unsigned lt_mask = (1u << lane) - 1u;
    uint32_t *wh = whist + warp * kBins;

    for (int64_t tile0 = begin; tile0 < end; tile0 += TILE) {
        const int valid = (int)((end - tile0) < TILE ? (end - tile0) : TILE);
        for (int i = threadIdx.x; i < kWarps * kBins; i += kBlock) whist[i] = 0;
        __syncthreads();
        K k[ITEMS];
        uint32_t v[ITEMS];
        int dg[ITEMS];
        uint32_t rk[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            // warp-striped: stable order inside the tile is (warp, j, lane)
            const int idx = warp * (32 * ITEMS) + j * 32 + lane;
            if (idx < valid) {
                k[j] = keys_in[tile0 + idx];
                v[j] = HasVals ? vals_in[tile0 + idx] : 0u;
                dg[j] = digit_of(k[j], shift, mask);
            } else {
                k[j] = ~K(0);
                v[j] = 0u;
                dg[j] = kBins - 1;  // padding ranks last in the last bucket
            }
        }
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const unsigned peers = __match_any_sync(0xffffffffu, dg[j]);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (lane == leader) {
                base = wh[dg[j]];
                wh[dg[j]] = base + (uint32_t)__popc(peers);
            }
            base = __shfl_sync(0xffffffffu, base, leader);
            rk[j] = base + (uint32_t)__popc(peers & lt_mask);
            __syncwarp();
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kBins; d += kBlock) {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = whist[w * kBins + d];
                whist[w * kBins + d] = s;
                s += c;
            }
            tcount[d] = s;
        }
        __syncthreads();
        int64_t tot;
        const int64_t ex = block_exclusive_sum<kBlock>((int64_t)tcount[threadIdx.x], scan_tmp, &tot);
        tstart[threadIdx.x] = (uint32_t)ex;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t pos = tstart[dg[j]] + wh[dg[j]] + rk[j];
            skeys[pos] = k[j];
            if (HasVals) svals[pos] = v[j];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < valid; i += kBlock) {
            const K kk = skeys[i];
            const int d = digit_of(kk, shift, mask);
            const uint32_t dst = running[d] + ((uint32_t)i - tstart[d]);
            keys_out[dst] = kk;
            if (HasVals) vals_out[dst] = svals[i];
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kBins; d += kBlock) {
            uint32_t c = tcount[d];
            if (d == kBins - 1) c -= (uint32_t)(TILE - valid);
            running[d] += c;
        }
        __syncthreads();
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
int downsweep_smem_bytes() {
    constexpr int TILE = kBlock * SortTraits<K>::kItems;
    return TILE * (int)sizeof(K) + (HasVals ? TILE * 4 : 0) + (kWarps * kBins + 3 * kBins) * 4;
}

template <class K>
int radix_sort_impl(K *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit, cudaStream_t st,
                    const char *timer_name) {
    if (n < 0) return set_error(GSMAT_ERR_INVALID_ARG, "radix sort: negative n");
    if (begin_bit < 0 || end_bit > (int)(8 * sizeof(K)) || begin_bit > end_bit) {
        return set_error(GSMAT_ERR_INVALID_ARG, "radix sort: bad bit range [%d,%d)", begin_bit, end_bit);
    }
    if (n <= 1 || begin_bit == end_bit) return GSMAT_OK;
    if (n > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "radix sort: n = %lld >= 2^32", (long long)n);
    constexpr int TILE = kBlock * SortTraits<K>::kItems;
    const int64_t ntiles = (n + TILE - 1) / TILE;
    int64_t ctas = (int64_t)sm_count() * 4;
    if (ctas > ntiles) ctas = ntiles;
    const int64_t tiles_per_cta = (ntiles + ctas - 1) / ctas;
    const int64_t span = tiles_per_cta * TILE;
    const int num_ctas = (int)((n + span - 1) / span);

    DevBuf alt_k, alt_v, counts;
    GS_TRY(alt_k.alloc(sizeof(K) * (size_t)n, st));
    if (vals) GS_TRY(alt_v.alloc(sizeof(uint32_t) * (size_t)n, st));
    GS_TRY(counts.alloc(sizeof(uint32_t) * (size_t)kBins * num_ctas, st));

    const int smem = vals ? downsweep_smem_bytes<K, true>() : downsweep_smem_bytes<K, false>();
    static bool attr_set[2] = {false, false};
    if (!attr_set[vals ? 1 : 0]) {
        if (vals) {
            GS_CUDA(cudaFuncSetAttribute(radix_downsweep<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        } else {
            GS_CUDA(cudaFuncSetAttribute(radix_downsweep<K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        }
        attr_set[vals ? 1 : 0] = true;
    }

    K *src_k = keys, *dst_k = alt_k.as<K>();
    uint32_t *src_v = vals, *dst_v = alt_v.as<uint32_t>();
    const int n_pass = (end_bit - begin_bit + 7) / 8;
    KernelTimer t(timer_name, st, (double)n * (2.0 * sizeof(K) + (vals ? 8.0 : 0.0)) * n_pass, (double)n);
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        const int width = end_bit - shift < 8 ? end_bit - shift : 8;
        const int mask = (1 << width) - 1;
        radix_upsweep<K><<<num_ctas, kBlock, 0, st>>>(src_k, n, span, shift, mask, num_ctas, counts.as<uint32_t>());
        GS_TRY(exclusive_scan_u32_inplace(counts.as<uint32_t>(), (int64_t)kBins * num_ctas, st));
        if (vals) {
            radix_downsweep<K, true><<<num_ctas, kBlock, smem, st>>>(src_k, src_v, dst_k, dst_v, n, span, shift, mask,
                                                                     num_ctas, counts.as<uint32_t>());
        } else {
            radix_downsweep<K, false><<<num_ctas, kBlock, smem, st>>>(src_k, nullptr, dst_k, nullptr, n, span, shift,
                                                                      mask, num_ctas, counts.as<uint32_t>());
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

int radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit, cudaStream_t st) {
    return radix_sort_impl<uint64_t>(keys, vals, n, begin_bit, end_bit, st, "radix_sort_u64");
}

int radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit, cudaStream_t st) {
    return radix_sort_impl<uint32_t>(keys, vals, n, begin_bit, end_bit, st, "radix_sort_u32");
}

int device_sm_count() { return sm_count(); }

}  // namespace gs
