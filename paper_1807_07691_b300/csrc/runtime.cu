// Process-wide runtime of libgsmat: error records, the allocator hook,
// pinned host scratch and the kernel-timing registry.
#include <stdarg.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>

#include "common.cuh"

namespace gs {

// ---------------------------------------------------------------------------
// errors

static thread_local std::string t_last_error;

int set_error(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return status;
}

void clear_error() { t_last_error.clear(); }

const char *last_error() { return t_last_error.c_str(); }

// ---------------------------------------------------------------------------
// allocator hook

static std::mutex g_alloc_mu;
static gsmat_alloc_fn g_alloc = nullptr;
static gsmat_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;
static bool g_pool_configured[64] = {false};  // guarded by g_alloc_mu

static void configure_default_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    if (g_pool_configured[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        // keep freed blocks in the pool instead of returning them at every sync
        uint64_t threshold = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
    }
    g_pool_configured[dev] = true;
}

void *dev_alloc_raw(size_t bytes, cudaStream_t st) {
    gsmat_alloc_fn a;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        ctx = g_alloc_ctx;
        if (!a) configure_default_pool();
    }
    // 256-byte alignment is guaranteed by both cudaMallocAsync and the
    // documented contract of the hook.
    if (a) return a(bytes, ctx, (gsmat_stream_t)st);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free_raw(void *p, cudaStream_t st) {
    if (!p) return;
    gsmat_free_fn f;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        f = g_free;
        ctx = g_alloc_ctx;
    }
    if (f) {
        f(p, ctx, (gsmat_stream_t)st);
        return;
    }
    cudaFreeAsync(p, st);
}

int set_allocator(gsmat_alloc_fn a, gsmat_free_fn f, void *ctx) {
    if ((a == nullptr) != (f == nullptr)) {
        return set_error(GSMAT_ERR_INVALID_ARG, "alloc and free must both be set or both be NULL");
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = a;
    g_free = f;
    g_alloc_ctx = a ? ctx : nullptr;
    return GSMAT_OK;
}

// ---------------------------------------------------------------------------
// pinned host scratch

// Mapped (device-addressable) pinned memory, one buffer per host thread, so
// that kernels can read small inputs from it and write small results into
// it without the copy engines (a small read-back queued behind a large
// device-to-host copy on another stream would wait for that copy).
struct ScratchHolder {
    int64_t *p = nullptr;
    int64_t *d = nullptr;
    int cap = 0;
    ~ScratchHolder() {
        if (p) cudaFreeHost(p);
    }
};
static thread_local ScratchHolder t_scratch;

int64_t *pinned_scratch(int n_words) {
    ScratchHolder &h = t_scratch;
    if (h.cap < n_words) {
        if (h.p) cudaFreeHost(h.p);
        h.p = h.d = nullptr;
        h.cap = 0;
        // one size for every use in practice (a re-allocation synchronises)
        int cap = n_words < 1024 ? 1024 : n_words;
        if (cudaHostAlloc((void **)&h.p, sizeof(int64_t) * (size_t)cap, cudaHostAllocMapped | cudaHostAllocPortable) !=
                cudaSuccess ||
            cudaHostGetDevicePointer((void **)&h.d, h.p, 0) != cudaSuccess) {
            cudaGetLastError();
            if (h.p) cudaFreeHost(h.p);
            h.p = h.d = nullptr;
            return nullptr;
        }
        h.cap = cap;
    }
    return h.p;
}

void *pinned_scratch_device(const void *host_ptr) {
    const ScratchHolder &h = t_scratch;
    const char *hp = static_cast<const char *>(host_ptr);
    const char *base = reinterpret_cast<const char *>(h.p);
    if (!h.p || hp < base || hp >= base + sizeof(int64_t) * (size_t)h.cap) return nullptr;
    return reinterpret_cast<char *>(h.d) + (hp - base);
}

// dst[0..n) = src[0..n), then (after a system-scope fence) dst[n] = tag.
__global__ void copy_words_kernel(const int64_t *__restrict__ src, int64_t *__restrict__ dst, int n, int64_t tag) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    __syncwarp();
    if (threadIdx.x == 0) {
        __threadfence_system();
        *(volatile int64_t *)(dst + n) = tag;
    }
}

// The copy kernel is the last work on the stream, so once its tag is in
// host memory everything before it has finished: the host spins on the tag
// (faster to wake than a stream synchronisation), asking the stream every
// 1024 spins so that an error or a lost tag ends the wait.
static int spin_on_tag(volatile int64_t *tag, int64_t want, cudaStream_t st) {
    for (uint64_t spin = 1; *tag != want; ++spin) {
        if ((spin & 1023) == 0) {
            const cudaError_t q = cudaStreamQuery(st);
            if (q == cudaSuccess) {
                if (*tag == want) break;
                return set_error(GSMAT_ERR_CUDA, "stream idle but the completion tag is missing");
            }
            if (q != cudaErrorNotReady) return set_error(GSMAT_ERR_CUDA, "stream wait: %s", cudaGetErrorString(q));
        }
#if defined(__x86_64__)
        __builtin_ia32_pause();
#endif
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    return GSMAT_OK;
}

static thread_local int64_t t_tag_seq = 0;

int read_words(const void *d_src, int64_t *h_dst, int n_words, cudaStream_t st) {
    void *d_dst = pinned_scratch_device(h_dst);
    if (!d_dst || !pinned_scratch_device(h_dst + n_words)) {
        return set_error(GSMAT_ERR_INVALID_ARG, "read_words: destination outside the pinned scratch");
    }
    const int64_t want = ++t_tag_seq;
    volatile int64_t *tag = h_dst + n_words;
    *tag = 0;
    copy_words_kernel<<<1, 32, 0, st>>>(static_cast<const int64_t *>(d_src), static_cast<int64_t *>(d_dst), n_words,
                                        want);
    GS_LAUNCH_CHECK();
    return spin_on_tag(tag, want, st);
}

int wait_stream(cudaStream_t st) {
    int64_t *h = pinned_scratch(kScratchTagWord + 1);
    if (!h) return set_error(GSMAT_ERR_CUDA, "pinned host scratch");
    const int64_t want = ++t_tag_seq;
    volatile int64_t *tag = h + kScratchTagWord;
    *tag = 0;
    copy_words_kernel<<<1, 32, 0, st>>>(nullptr, static_cast<int64_t *>(pinned_scratch_device(h + kScratchTagWord)), 0,
                                        want);
    GS_LAUNCH_CHECK();
    return spin_on_tag(tag, want, st);
}

// ---------------------------------------------------------------------------
// kernel timing

struct ProfAgg {
    int64_t launches = 0;
    double ms = 0, bytes = 0, items = 0;
};

static std::mutex g_prof_mu;
static std::map<std::string, ProfAgg> g_prof;
static std::atomic<bool> g_prof_on{false};

struct PendingTimer {
    const char *name;
    cudaEvent_t a, b;
    double bytes, items;
    bool counts;  // counts as a call (false: a later segment of the same call)
};
static thread_local std::vector<PendingTimer> t_pending;
static thread_local std::vector<cudaEvent_t> t_event_pool;

static cudaEvent_t get_event() {
    if (!t_event_pool.empty()) {
        cudaEvent_t e = t_event_pool.back();
        t_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

bool profile_on() { return g_prof_on.load(std::memory_order_relaxed); }

KernelTimer::KernelTimer(const char *n, cudaStream_t s, double algo_bytes, double n_items, bool counts_call)
    : name(n), st(s), bytes(algo_bytes), items(n_items), counts(counts_call) {
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    a = get_event();
    b = get_event();
    if (!a || !b) {
        a = b = nullptr;
        return;
    }
    cudaEventRecord(a, st);
}

void KernelTimer::stop() {
    if (!a) return;
    cudaEventRecord(b, st);
    t_pending.push_back({name, a, b, bytes, items, counts});
    a = b = nullptr;
}

void profile_flush() {
    if (t_pending.empty()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &p : t_pending) {
        float ms = 0;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            auto &g = g_prof[p.name];
            if (p.counts) g.launches++;
            g.ms += ms;
            g.bytes += p.bytes;
            g.items += p.items;
        } else {
            cudaGetLastError();
        }
        t_event_pool.push_back(p.a);
        t_event_pool.push_back(p.b);
    }
    t_pending.clear();
}

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

int profile_enable(int on) {
    g_prof_on.store(on != 0, std::memory_order_relaxed);
    return GSMAT_OK;
}

int profile_read(gsmat_kernel_profile *out, int32_t cap, int32_t *n_out, int reset) {
    profile_flush();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int32_t n = 0;
    for (auto &kv : g_prof) {
        if (out && n < cap) {
            gsmat_kernel_profile &o = out[n];
            memset(&o, 0, sizeof(o));
            strncpy(o.name, kv.first.c_str(), sizeof(o.name) - 1);
            o.launches = kv.second.launches;
            o.total_ms = kv.second.ms;
            o.algo_bytes = kv.second.bytes;
            o.items = kv.second.items;
        }
        n++;
    }
    if (n_out) *n_out = n;
    if (reset) g_prof.clear();
    return GSMAT_OK;
}

}  // namespace gs
