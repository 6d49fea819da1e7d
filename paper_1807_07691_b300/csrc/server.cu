// Continuous-batching request server over a resident store.
//
// Requests (one BGP each) are submitted from any host thread and return a
// ticket at once.  A scheduler thread admits queued requests, in arrival
// order, into a micro-batch whenever one of `slots` in-flight slots is free
// and the requests' estimated intermediate bytes (the planner's accumulated
// estimate of Sec. 6.2 times the row width) fit in the device budget still
// unclaimed; each micro-batch is planned and launched on its own stream, so
// requests that arrive while others are on the GPU start as soon as a slot
// and memory free up, and their work overlaps on the device.  A completion
// thread finishes micro-batches as their device work ends (in whatever
// order), stamps every request's latency and releases its budget.  Each
// result is the one the plain path gives for that BGP alone.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "plan.h"
#include "query.cuh"
#include "store.cuh"

namespace gs {
int batch_prepare_with(const gsmat_store *S, const gsmat_bgp *bgps, int32_t n, const gsmat_batch_config *cfg,
                       cudaStream_t st, const BatchResources *res, gsmat_batch **out);
int batch_launch_async(gsmat_batch *B);
int batch_finish(gsmat_batch *B);
int batch_kernel_done(gsmat_batch *B);
void batch_free(gsmat_batch *B);
int batch_result_view(const gsmat_batch *B, int32_t i, int64_t *rows, int32_t *cols, const int32_t **col_ptrs);
int batch_result(const gsmat_batch *B, int32_t i, int64_t *rows, int32_t *cols, int32_t *path);
int batch_copy(const gsmat_batch *B, int32_t i, int32_t *dst, int dst_on_device, cudaStream_t st);
}  // namespace gs

namespace {

using Clock = std::chrono::steady_clock;

struct BatchHolder {
    gsmat_batch *B = nullptr;
    ~BatchHolder() {
        if (B) gs::batch_free(B);
    }
};

// A result of the plain path (a request admitted alone).
struct TableHolder {
    gsmat_table *T = nullptr;
    ~TableHolder() { delete T; }
};

enum { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_FAILED = 3 };

struct Request {
    int64_t ticket = 0;
    std::vector<gsmat_pattern> pats;
    int n_vars = 0;
    double est_bytes = 0;
    int state = REQ_QUEUED;
    int status = GSMAT_OK;
    Clock::time_point t_submit, t_done;
    std::shared_ptr<BatchHolder> batch;  // result in a micro-batch ...
    int index = -1;
    std::shared_ptr<TableHolder> table;  // ... or of the plain path
};

struct InFlight {
    std::shared_ptr<BatchHolder> holder;
    std::vector<std::shared_ptr<Request>> reqs;
    double bytes = 0;
    int slot = -1;
};

}  // namespace

struct gsmat_server {
    const gsmat_store *S = nullptr;
    gsmat_server_config cfg{};
    int device = 0;
    cudaStream_t prep_stream = nullptr;
    std::mutex mu;
    std::condition_variable cv_sched, cv_comp, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<int64_t, std::shared_ptr<Request>> reqs;
    std::deque<InFlight> inflight;
    std::vector<gs::BatchResources> res;  // one set per slot, reused by its micro-batches
    std::vector<int> free_slots;
    int64_t next_ticket = 1;
    double inflight_bytes = 0;
    int launching = 0;  // micro-batches being planned (hold a slot)
    uint64_t finished_batches = 0;
    bool stop = false;
    bool sched_done = false;  // the scheduler has exited (nothing more will be launched)
    gsmat_server_stats_t stats{};
    // direct lanes: each runs one request at a time on the plain path (as
    // gsmat_query), on its own stream and thread, while the scheduler keeps
    // admitting micro-batches
    struct Lane {
        cudaStream_t st = nullptr;
        std::shared_ptr<Request> req;  // handed over, not yet finished (under mu)
        double bytes = 0;
        std::atomic<int> pending{0};   // 1 while req is set (read without the lock)
        std::thread th;
    };
    std::vector<std::unique_ptr<Lane>> lanes;
    std::condition_variable cv_lane;
    std::atomic<uint64_t> submit_seq{0};  // submissions so far (read without the lock)
    std::thread sched, comp;
};

namespace gs {
namespace {

// Estimated device bytes of one request: the plan's accumulated estimate
// (Sec. 6.2) with constant rows taken at their predicate's average row size,
// times the widest row, for tables and their temporaries.
double estimate_bytes(const gsmat_store *S, const gsmat_pattern *pats, int n, int n_vars, bool plan_cost) {
    std::vector<int64_t> keys(n);
    std::vector<gsmat_pred_stats> st(n);
    for (int i = 0; i < n; ++i) {
        memset(&st[i], 0, sizeof(st[i]));
        const int32_t sl = S->slot_of(pats[i].p);
        if (sl < 0) return 4096.0;  // empty result
        st[i].nnz = S->side[0][sl].nnz;
        st[i].nr_s = S->side[0][sl].nrows;
        st[i].nr_o = S->side[1][sl].nrows;
        const double avg_s = st[i].nr_s ? (double)st[i].nnz / st[i].nr_s : 0.0;
        const double avg_o = st[i].nr_o ? (double)st[i].nnz / st[i].nr_o : 0.0;
        if (!pats[i].s_var && !pats[i].o_var) keys[i] = 1;
        else if (!pats[i].s_var) keys[i] = (int64_t)(avg_s + 1.0);
        else if (!pats[i].o_var) keys[i] = (int64_t)(avg_o + 1.0);
        else keys[i] = st[i].nnz;
    }
    std::vector<int32_t> order(n), kinds(n);
    std::vector<double> est(n);
    if ((plan_cost ? plan_bgp_cost : plan_bgp)(pats, n, keys.data(), st.data(), order.data(), kinds.data(),
                                               est.data()) != GSMAT_OK) {
        return 1e12;
    }
    double total = 0;
    for (double e : est) total += e;
    return 4096.0 + total * 4.0 * std::max(1, n_vars) * 2.0;
}

void fail_requests(gsmat_server *srv, std::vector<std::shared_ptr<Request>> &rs, int status) {
    const Clock::time_point now = Clock::now();
    for (auto &r : rs) {
        r->state = REQ_FAILED;
        r->status = status;
        r->t_done = now;
        srv->stats.failed++;
    }
}

// Wait-loop pause of the threads that spin before blocking.
inline void cpu_relax() {
#if defined(__x86_64__)
    __builtin_ia32_pause();
#else
    std::this_thread::yield();
#endif
}

// The scheduler and the direct lanes spin this long on their next event
// before blocking on a condition variable: at a few hundred requests per
// second and more they never sleep, so a request is not delayed by a thread
// wake-up (tens of microseconds each); below that they block.
constexpr int kSpinUs = 2000;

// A direct lane: runs each handed-over request on the plain path (as
// gsmat_query) on its own stream, then completes it.  The scheduler hands a
// request to an idle lane when it found the queue empty, so under light load
// every request starts at once on the plain path's multi-CTA steps (a
// one-query micro-batch runs on one CTA and pays the batch machinery);
// requests that queue up behind busy lanes form micro-batches.
void lane_loop(gsmat_server *srv, gsmat_server::Lane *L) {
    cudaSetDevice(srv->device);
    while (true) {
        {
            const Clock::time_point until = Clock::now() + std::chrono::microseconds(kSpinUs);
            while (!L->pending.load(std::memory_order_acquire) && Clock::now() < until) cpu_relax();
        }
        std::shared_ptr<Request> r;
        double bytes = 0;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_lane.wait(lk, [&] { return srv->sched_done || L->req != nullptr; });
            if (!L->req) return;  // the scheduler is gone and nothing is pending
            r = L->req;
            bytes = L->bytes;
        }
        auto holder = std::make_shared<TableHolder>();
        const uint32_t flags = srv->cfg.batch.plan_cost ? GSMAT_PLAN_COST : GSMAT_SORTED;
        const int rc = query_run(srv->S, r->pats.data(), (int)r->pats.size(), r->n_vars, flags, L->st, &holder->T);
        profile_flush();
        const Clock::time_point now = Clock::now();
        std::lock_guard<std::mutex> lk(srv->mu);
        L->req = nullptr;
        L->pending.store(0, std::memory_order_release);
        srv->inflight_bytes -= bytes;
        srv->finished_batches++;
        r->t_done = now;
        if (rc == GSMAT_OK) {
            r->table = std::move(holder);
            r->state = REQ_DONE;
            srv->stats.completed++;
            srv->stats.direct++;
        } else {
            r->state = REQ_FAILED;
            r->status = rc;
            srv->stats.failed++;
        }
        srv->cv_done.notify_all();
        srv->cv_sched.notify_all();
    }
}

void scheduler_loop(gsmat_server *srv) {
    cudaSetDevice(srv->device);
    while (true) {
        std::vector<std::shared_ptr<Request>> take;
        double bytes = 0;
        int slot = -1;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            auto idle_lane = [&]() -> gsmat_server::Lane * {
                for (auto &L : srv->lanes) {
                    if (!L->req) return L.get();
                }
                return nullptr;
            };
            // a slot is free only once the completion thread has finished
            // its micro-batch and handed the slot's resources back
            auto ready = [&] {
                return srv->stop ||
                       (!srv->queue.empty() && (!srv->free_slots.empty() || (srv->queue.size() == 1 && idle_lane())));
            };
            if (!ready()) {
                // spin on the submissions before blocking (see kSpinUs)
                const uint64_t seen = srv->submit_seq.load(std::memory_order_acquire);
                lk.unlock();
                const Clock::time_point until = Clock::now() + std::chrono::microseconds(kSpinUs);
                while (srv->submit_seq.load(std::memory_order_acquire) == seen && Clock::now() < until) cpu_relax();
                lk.lock();
                srv->cv_sched.wait(lk, ready);
            }
            if (srv->stop) {
                std::vector<std::shared_ptr<Request>> rest(srv->queue.begin(), srv->queue.end());
                srv->queue.clear();
                fail_requests(srv, rest, GSMAT_ERR_INVALID_ARG);
                srv->sched_done = true;
                srv->cv_done.notify_all();
                srv->cv_comp.notify_all();
                srv->cv_lane.notify_all();
                return;
            }
            // a request that found the queue empty goes to an idle direct lane
            if (srv->queue.size() == 1) {
                gsmat_server::Lane *L = idle_lane();
                const double b = srv->queue.front()->est_bytes;
                const bool fits = srv->inflight_bytes + b <= (double)srv->cfg.budget_bytes;
                if (L && (fits || (srv->inflight.empty() && srv->launching == 0 && srv->inflight_bytes == 0))) {
                    std::shared_ptr<Request> r = srv->queue.front();
                    srv->queue.pop_front();
                    srv->inflight_bytes += b;
                    r->state = REQ_RUNNING;
                    L->req = r;
                    L->bytes = b;
                    L->pending.store(1, std::memory_order_release);
                    srv->cv_lane.notify_all();
                    continue;
                }
                if (srv->free_slots.empty()) {
                    // the lane cannot take it yet (budget) and no slot is free
                    const uint64_t seen = srv->finished_batches;
                    srv->cv_sched.wait(lk, [&] { return srv->stop || srv->finished_batches != seen; });
                    continue;
                }
            }
            // admission: arrival order, under the budget; a request larger
            // than the whole budget runs alone when nothing else is in flight
            bool lanes_busy = false;
            for (auto &L : srv->lanes) lanes_busy = lanes_busy || L->req != nullptr;
            while (!srv->queue.empty() && (int)take.size() < srv->cfg.max_batch) {
                const double b = srv->queue.front()->est_bytes;
                const bool fits = srv->inflight_bytes + bytes + b <= (double)srv->cfg.budget_bytes;
                const bool alone = take.empty() && srv->inflight.empty() && srv->launching == 0 && !lanes_busy;
                if (!fits && !alone) break;
                take.push_back(srv->queue.front());
                srv->queue.pop_front();
                bytes += b;
                if (!fits) break;
            }
            if (take.empty()) {
                // budget exhausted: wait for a micro-batch to finish
                const uint64_t seen = srv->finished_batches;
                srv->cv_sched.wait(lk, [&] { return srv->stop || srv->finished_batches != seen; });
                continue;
            }
            srv->inflight_bytes += bytes;
            srv->launching++;
            for (auto &r : take) r->state = REQ_RUNNING;
            slot = srv->free_slots.back();  // non-empty: checked by the wait above, under the same lock
            srv->free_slots.pop_back();
        }
        std::vector<gsmat_bgp> bgps(take.size());
        for (size_t i = 0; i < take.size(); ++i) {
            bgps[i].pats = take[i]->pats.data();
            bgps[i].n_pats = (int32_t)take[i]->pats.size();
            bgps[i].n_vars = take[i]->n_vars;
        }
        gsmat_batch_config bc = srv->cfg.batch;
        bc.use_graph = 0;        // one run per micro-batch: launch directly
        bc.compact_results = 1;  // results outlive the arena, which is released at once
        const int64_t want = (int64_t)std::min<double>(4.0 * bytes, (double)srv->cfg.batch.arena_bytes);
        bc.arena_bytes = std::max<int64_t>(want, std::min<int64_t>((int64_t)256 << 20, srv->cfg.batch.arena_bytes));
        auto holder = std::make_shared<BatchHolder>();
        int rc = batch_prepare_with(srv->S, bgps.data(), (int32_t)bgps.size(), &bc, srv->prep_stream, &srv->res[slot],
                                    &holder->B);
        if (rc == GSMAT_OK) rc = batch_launch_async(holder->B);
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->launching--;
        if (rc != GSMAT_OK) {
            srv->free_slots.push_back(slot);
            srv->inflight_bytes -= bytes;
            fail_requests(srv, take, rc);
            srv->cv_done.notify_all();
            srv->cv_sched.notify_all();
            continue;
        }
        for (size_t i = 0; i < take.size(); ++i) {
            take[i]->batch = holder;
            take[i]->index = (int)i;
        }
        srv->stats.batches++;
        srv->inflight.push_back(InFlight{holder, std::move(take), bytes, slot});
        srv->cv_comp.notify_all();
    }
}

void completion_loop(gsmat_server *srv) {
    cudaSetDevice(srv->device);
    while (true) {
        InFlight job;
        bool have = false;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            // exit only once the scheduler is gone and nothing is in flight:
            // a micro-batch being planned when stop is set still arrives
            srv->cv_comp.wait(lk, [&] { return srv->sched_done || !srv->inflight.empty(); });
            if (srv->inflight.empty() && srv->sched_done) return;
            // the first micro-batch whose device work has ended
            for (auto it = srv->inflight.begin(); it != srv->inflight.end(); ++it) {
                if (batch_kernel_done(it->holder->B)) {
                    job = std::move(*it);
                    srv->inflight.erase(it);
                    have = true;
                    break;
                }
            }
        }
        if (!have) {
            // a dedicated thread: wait 5 us by the clock, yielding, before
            // the next look (a timed sleep adds the timer's slack, tens of
            // microseconds, to every request's latency; the pause keeps the
            // lock free for the submitters)
            const Clock::time_point until = Clock::now() + std::chrono::microseconds(5);
            while (Clock::now() < until) std::this_thread::yield();
            continue;
        }
        const int rc = batch_finish(job.holder->B);
        profile_flush();
        const Clock::time_point now = Clock::now();
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->inflight_bytes -= job.bytes;
        srv->finished_batches++;
        srv->free_slots.push_back(job.slot);  // the batch keeps only device memory and host vectors
        for (auto &r : job.reqs) {
            if (rc == GSMAT_OK) {
                r->state = REQ_DONE;
                r->t_done = now;
                srv->stats.completed++;
                int32_t path = 0;
                if (batch_result(job.holder->B, r->index, nullptr, nullptr, &path) == GSMAT_OK && path == 1) {
                    srv->stats.fallbacks++;
                }
            } else {
                r->state = REQ_FAILED;
                r->status = rc;
                r->t_done = now;
                srv->stats.failed++;
            }
        }
        srv->cv_done.notify_all();
        srv->cv_sched.notify_all();
    }
}

std::shared_ptr<Request> find(gsmat_server *srv, int64_t ticket) {
    auto it = srv->reqs.find(ticket);
    return it == srv->reqs.end() ? nullptr : it->second;
}

}  // namespace

void server_destroy(gsmat_server *srv);

int server_create(const gsmat_store *S, const gsmat_server_config *cfg, gsmat_server **out) {
    if (!S || !out) return set_error(GSMAT_ERR_INVALID_ARG, "store or out is NULL");
    *out = nullptr;
    gsmat_server *srv = new gsmat_server();
    srv->S = S;
    gsmat_server_config c;
    memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    if (c.max_batch <= 0) c.max_batch = 1024;
    if (c.slots <= 0) c.slots = 4;
    if (c.budget_bytes <= 0) c.budget_bytes = (int64_t)120 << 30;
    if (c.batch.block == 0) c.batch.block = 512;
    if (c.batch.ctas_per_sm == 0) c.batch.ctas_per_sm = 1;
    if (c.batch.arena_bytes == 0) c.batch.arena_bytes = (int64_t)8 << 30;
    if (c.lanes <= 0) c.lanes = 2;
    if (c.slots > 64 || c.max_batch > (1 << 20) || c.lanes > 64) {
        delete srv;
        return set_error(GSMAT_ERR_INVALID_ARG, "server slots or max_batch out of range");
    }
    if (c.batch.plan_cost != 0 && c.batch.plan_cost != 1) {
        delete srv;
        return set_error(GSMAT_ERR_INVALID_ARG, "bad batch plan_cost %d (0 or 1)", c.batch.plan_cost);
    }
    srv->cfg = c;
    cudaGetDevice(&srv->device);
    if (cudaStreamCreateWithFlags(&srv->prep_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete srv;
        return set_error(GSMAT_ERR_CUDA, "server stream");
    }
    const int n_lanes = c.batch_lone ? 0 : c.lanes;
    for (int k = 0; k < n_lanes; ++k) {
        srv->lanes.push_back(std::make_unique<gsmat_server::Lane>());
        if (cudaStreamCreateWithFlags(&srv->lanes.back()->st, cudaStreamNonBlocking) != cudaSuccess) {
            srv->lanes.back()->st = nullptr;
            server_destroy(srv);
            return set_error(GSMAT_ERR_CUDA, "server lane stream");
        }
    }
    srv->res.resize(c.slots);
    for (int k = 0; k < c.slots; ++k) {
        BatchResources &r = srv->res[k];
        memset(&r, 0, sizeof(r));
        bool ok = cudaStreamCreateWithFlags(&r.st, cudaStreamNonBlocking) == cudaSuccess;
        for (int e = 0; e < 4 && ok; ++e) ok = cudaEventCreate(&r.ev[e]) == cudaSuccess;
        ok = ok && cudaMallocHost((void **)&r.results_host, sizeof(BResult) * (size_t)c.max_batch) == cudaSuccess;
        ok = ok && cudaMallocHost((void **)&r.ctrl_host, 2 * sizeof(unsigned long long)) == cudaSuccess;
        r.cap = c.max_batch;
        srv->free_slots.push_back(k);
        if (!ok) {
            server_destroy(srv);
            return set_error(GSMAT_ERR_CUDA, "server slot resources");
        }
    }
    srv->sched = std::thread(scheduler_loop, srv);
    srv->comp = std::thread(completion_loop, srv);
    for (auto &L : srv->lanes) L->th = std::thread(lane_loop, srv, L.get());
    *out = srv;
    return GSMAT_OK;
}

int server_submit(gsmat_server *srv, const gsmat_pattern *pats, int n_pats, int n_vars, int64_t *ticket) {
    if (!srv || !ticket) return set_error(GSMAT_ERR_INVALID_ARG, "server or ticket is NULL");
    GS_TRY(validate_bgp(pats, n_pats, n_vars));
    auto r = std::make_shared<Request>();
    r->pats.assign(pats, pats + n_pats);
    r->n_vars = n_vars;
    r->est_bytes = estimate_bytes(srv->S, pats, n_pats, n_vars, srv->cfg.batch.plan_cost != 0);
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return set_error(GSMAT_ERR_INVALID_ARG, "server is shutting down");
    r->ticket = srv->next_ticket++;
    srv->reqs[r->ticket] = r;
    srv->queue.push_back(r);
    srv->stats.submitted++;
    *ticket = r->ticket;
    srv->submit_seq.fetch_add(1, std::memory_order_release);
    srv->cv_sched.notify_one();
    return GSMAT_OK;
}

int server_wait(gsmat_server *srv, int64_t ticket, int64_t timeout_us, int32_t *done) {
    if (!srv) return set_error(GSMAT_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto r = find(srv, ticket);
    if (!r) return set_error(GSMAT_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
    auto ready = [&] { return r->state >= REQ_DONE; };
    if (timeout_us < 0) {
        srv->cv_done.wait(lk, ready);
    } else {
        srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    if (done) *done = r->state >= REQ_DONE ? 1 : 0;
    if (r->state == REQ_FAILED) return set_error(r->status, "request %lld failed", (long long)ticket);
    return GSMAT_OK;
}

int server_result(gsmat_server *srv, int64_t ticket, int64_t *rows, int32_t *cols, double *latency_us) {
    if (!srv) return set_error(GSMAT_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto r = find(srv, ticket);
    if (!r) return set_error(GSMAT_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
    if (r->state == REQ_FAILED) return set_error(r->status, "request %lld failed", (long long)ticket);
    if (r->state != REQ_DONE) return set_error(GSMAT_ERR_INVALID_ARG, "request %lld not finished", (long long)ticket);
    if (latency_us) {
        *latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    }
    if (r->table) {
        if (rows) *rows = r->table->T->rows;
        if (cols) *cols = r->table->T->ncols;
        return GSMAT_OK;
    }
    return batch_result_view(r->batch->B, r->index, rows, cols, nullptr);
}

int server_copy(gsmat_server *srv, int64_t ticket, int32_t *dst, int dst_on_device, cudaStream_t st) {
    std::shared_ptr<BatchHolder> holder;
    std::shared_ptr<TableHolder> table;
    int index;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto r = find(srv, ticket);
        if (!r || r->state != REQ_DONE) return set_error(GSMAT_ERR_INVALID_ARG, "ticket %lld has no result", (long long)ticket);
        holder = r->batch;
        table = r->table;
        index = r->index;
    }
    if (table) return table_copy(table->T, dst, dst_on_device, st);
    return batch_copy(holder->B, index, dst, dst_on_device, st);
}

int server_release(gsmat_server *srv, int64_t ticket) {
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->reqs.find(ticket);
        if (it == srv->reqs.end()) return set_error(GSMAT_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
        if (it->second->state < REQ_DONE) return set_error(GSMAT_ERR_INVALID_ARG, "request %lld still running", (long long)ticket);
        r = it->second;
        srv->reqs.erase(it);
    }
    r.reset();  // the micro-batch's memory goes with its last released request
    return GSMAT_OK;
}

int server_stats(gsmat_server *srv, gsmat_server_stats_t *s) {
    if (!srv || !s) return set_error(GSMAT_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *s = srv->stats;
    s->queued = (int64_t)srv->queue.size();
    s->in_flight = (int64_t)srv->inflight.size() + srv->launching;
    s->in_flight_bytes = (int64_t)srv->inflight_bytes;
    return GSMAT_OK;
}

void server_destroy(gsmat_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_sched.notify_all();
    srv->cv_comp.notify_all();
    if (srv->sched.joinable()) srv->sched.join();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->sched_done = true;  // also when the scheduler never started
    }
    // the completion thread and the direct lanes drain what they hold, then exit
    srv->cv_comp.notify_all();
    srv->cv_lane.notify_all();
    if (srv->comp.joinable()) srv->comp.join();
    for (auto &L : srv->lanes) {
        if (L->th.joinable()) L->th.join();
        if (L->st) {
            cudaStreamSynchronize(L->st);
            cudaStreamDestroy(L->st);
        }
    }
    srv->reqs.clear();
    for (BatchResources &r : srv->res) {
        if (r.st) cudaStreamSynchronize(r.st);
    }
    for (BatchResources &r : srv->res) {
        if (r.st) cudaStreamDestroy(r.st);
        for (int e = 0; e < 4; ++e) {
            if (r.ev[e]) cudaEventDestroy(r.ev[e]);
        }
        if (r.results_host) cudaFreeHost(r.results_host);
        if (r.ctrl_host) cudaFreeHost(r.ctrl_host);
    }
    if (srv->prep_stream) cudaStreamDestroy(srv->prep_stream);
    delete srv;
}

}  // namespace gs
