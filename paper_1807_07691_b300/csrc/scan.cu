// Single-pass exclusive prefix sum (decoupled look-back) and a generic
// stable selection of int32 values.  The scan is the offset computation of
// the pre-allocation step of the GPU join (Sec. 7.2.2, Alg. 4: P_i =
// P_{i-1} + N_{i-1}), done on the device in int64.
#include <mutex>

#include "common.cuh"
#include "select.cuh"

namespace gs {
namespace {

constexpr int kScanBlock = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

// Shared-memory index with one padding word per 32, so that a thread
// reading its kScanItems consecutive values hits distinct banks.
__device__ __forceinline__ int padded(int i) { return i + (i >> 5); }

template <class InT, class OutT, bool WriteTotal>
__global__ void __launch_bounds__(kScanBlock) scan_kernel(const InT *in, OutT *out, int64_t n, LookbackScratch ls) {
    // in and out may be the same array: a tile reads its inputs before the
    // look-back and writes its outputs after it
    __shared__ int tile_sm;
    __shared__ int64_t scan_sm[kScanBlock / 32 + 1];
    __shared__ int64_t prefix_sm;
    __shared__ InT stage[kScanTile + kScanTile / 32];
    const int tile = acquire_tile_id(ls, &tile_sm);
    const int64_t t0 = (int64_t)tile * kScanTile;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int idx = j * kScanBlock + threadIdx.x;
        const int64_t i = t0 + idx;
        stage[padded(idx)] = i < n ? in[i] : InT(0);
    }
    __syncthreads();
    InT v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = stage[padded(threadIdx.x * kScanItems + j)];
        s += (int64_t)v[j];
    }
    int64_t tot;
    const int64_t ex = block_exclusive_sum<kScanBlock>(s, scan_sm, &tot);
    const int64_t pre = tile_lookback(ls, tile, tot, &prefix_sm);
    int64_t run = pre + ex;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = t0 + threadIdx.x * kScanItems + j;
        if (i < n) out[i] = (OutT)run;
        run += (int64_t)v[j];
    }
    if (WriteTotal && tile == (int)gridDim.x - 1 && threadIdx.x == 0) out[n] = (OutT)(pre + tot);
}

struct SelectI32Op {
    const int32_t *in;
    const uint8_t *flags;
    int32_t *out;
    __device__ bool flag(int64_t i) const { return flags[i] != 0; }
    __device__ void emit(int64_t i, int64_t j) const { out[j] = in[i]; }
};

}  // namespace

int exclusive_scan_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t st, int *err_word) {
    if (n < 0 || (n > 0 && !in) || !out) return set_error(GSMAT_ERR_INVALID_ARG, "scan: bad arguments");
    if (n == 0) {
        GS_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
        return GSMAT_OK;
    }
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles > INT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "scan over %lld items", (long long)n);
    LookbackBuf lb;
    GS_TRY(lb.make(ntiles, st, err_word));
    KernelTimer t("scan_i32", st, (double)n * 12.0, (double)n);
    scan_kernel<int32_t, int64_t, true><<<(unsigned)ntiles, kScanBlock, 0, st>>>(in, out, n, lb.view);
    GS_LAUNCH_CHECK();
    t.stop();
    return GSMAT_OK;
}

int exclusive_scan_u32_inplace(uint32_t *data, int64_t n, cudaStream_t st) {
    if (n <= 0) return GSMAT_OK;
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles > INT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "scan over %lld items", (long long)n);
    LookbackBuf lb;
    GS_TRY(lb.make(ntiles, st));
    scan_kernel<uint32_t, uint32_t, false><<<(unsigned)ntiles, kScanBlock, 0, st>>>(data, data, n, lb.view);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

// ---------------------------------------------------------------------------
// Exclusive scan that allocates nothing (for callers that cannot allocate
// device memory).  Its scratch -- one descriptor per tile, the dynamic tile
// counter and an error word -- is this file-scope array, resident on every
// device that loads the library until the process exits.  Host code must not
// pass the array's name to a kernel (on the host it is only a stand-in);
// the device address is looked up once per device with
// cudaGetSymbolAddress and cached.

constexpr int64_t kNoAllocMaxTiles = 32768;  // 256 KB of tile descriptors
constexpr int64_t kNoAllocMaxItems = kNoAllocMaxTiles * kScanTile;  // 67,108,864
// [0, kNoAllocMaxTiles): tile descriptors; then 4 words: counter | error
static __device__ __align__(256) unsigned long long g_noalloc_scan_scratch[kNoAllocMaxTiles + 4];

namespace {

struct NoAllocSetup {
    std::mutex mu;
    unsigned long long *addr[64] = {nullptr};
};
NoAllocSetup &noalloc_setup() {
    static NoAllocSetup s;
    return s;
}

// Device address of the scratch array on the current device (set-up on the
// first call per device).
int noalloc_scratch_ptr(unsigned long long **out) {
    int dev = 0;
    GS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(GSMAT_ERR_CUDA, "device ordinal %d out of range", dev);
    NoAllocSetup &s = noalloc_setup();
    std::lock_guard<std::mutex> lk(s.mu);
    if (!s.addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scan_scratch);
        if (e != cudaSuccess || !p) {
            return set_error(GSMAT_ERR_CUDA, "cudaGetSymbolAddress of the scan scratch: %s", cudaGetErrorString(e));
        }
        s.addr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = s.addr[dev];
    return GSMAT_OK;
}

}  // namespace

int64_t exclusive_scan_i32_noalloc_max() { return kNoAllocMaxItems; }

int exclusive_scan_i32_noalloc(const int32_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    if (n < 0 || (n > 0 && !in) || !out) return set_error(GSMAT_ERR_INVALID_ARG, "scan: bad arguments");
    if (n > kNoAllocMaxItems) {
        return set_error(GSMAT_ERR_CAPACITY, "scan without allocation: n = %lld exceeds the maximum %lld",
                         (long long)n, (long long)kNoAllocMaxItems);
    }
    unsigned long long *scratch = nullptr;
    GS_TRY(noalloc_scratch_ptr(&scratch));
    if (n == 0) {
        GS_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
        return GSMAT_OK;
    }
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    // the array keeps the previous call's contents: clear the descriptors in
    // use and the counter / error words
    GS_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (size_t)ntiles, st));
    GS_CUDA(cudaMemsetAsync(scratch + kNoAllocMaxTiles, 0, sizeof(unsigned long long) * 4, st));
    LookbackScratch view;
    view.status = scratch;
    view.tile_counter = reinterpret_cast<unsigned int *>(scratch + kNoAllocMaxTiles);
    view.error = reinterpret_cast<int *>(scratch + kNoAllocMaxTiles + 1);
    view.poll_limit = kLookbackPollLimit;
    scan_kernel<int32_t, int64_t, true><<<(unsigned)ntiles, kScanBlock, 0, st>>>(in, out, n, view);
    GS_LAUNCH_CHECK();
    return GSMAT_OK;
}

namespace {
__global__ void set_word_kernel(unsigned int *p, unsigned int v) { *p = v; }
}  // namespace

int selftest_wait_expiry(int poll_limit, cudaStream_t st) {
    if (poll_limit < 1 || poll_limit > kLookbackPollLimit) {
        return set_error(GSMAT_ERR_INVALID_ARG, "poll limit %d outside [1, %d]", poll_limit, kLookbackPollLimit);
    }
    constexpr int64_t kTiles = 4;
    const int64_t n = kTiles * kScanTile;
    DevBuf in, out, err;
    GS_TRY(in.alloc(sizeof(int32_t) * (size_t)n, st));
    GS_TRY(out.alloc(sizeof(int64_t) * (size_t)(n + 1), st));
    GS_TRY(err.alloc(sizeof(int64_t), st));  // an aligned word for read_words
    GS_CUDA(cudaMemsetAsync(in.p, 0, sizeof(int32_t) * (size_t)n, st));
    GS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int64_t), st));
    LookbackBuf lb;
    GS_TRY(lb.make(kTiles, st, err.as<int>()));
    lb.view.poll_limit = poll_limit;
    // The tile counter starts at 1: the kTiles - 1 CTAs take tiles 1..3 (all
    // inside the input), and tile 0's descriptor, which every look-back
    // window reaches, is never written.
    set_word_kernel<<<1, 1, 0, st>>>(lb.view.tile_counter, 1u);
    GS_LAUNCH_CHECK();
    scan_kernel<int32_t, int64_t, true><<<(unsigned)(kTiles - 1), kScanBlock, 0, st>>>(in.as<int32_t>(),
                                                                                      out.as<int64_t>(), n, lb.view);
    GS_LAUNCH_CHECK();
    int64_t *h = pinned_scratch(4);
    if (!h) return set_error(GSMAT_ERR_CUDA, "pinned host scratch");
    GS_TRY(read_words(err.p, h, 1, st));
    if ((int)h[0]) {
        return set_error(GSMAT_ERR_DEVICE_CHECK, "bounded wait expired (self-test: tile 0 never published)");
    }
    return GSMAT_OK;
}

int select_flagged_i32(const int32_t *in, const uint8_t *flags, int32_t *out, int64_t n, int64_t *d_count,
                       cudaStream_t st, int *err_word) {
    SelectI32Op op{in, flags, out};
    return run_select(op, n, d_count, st, err_word);
}

}  // namespace gs
