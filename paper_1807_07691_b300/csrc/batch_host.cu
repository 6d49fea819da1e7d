// Host side of batched evaluation: plans every BGP of a batch (Alg. 1) into
// a step program, uploads the programs, captures the device work (queue and
// arena reset, persistent kernel, result-descriptor copy) as a CUDA graph,
// and after each run finishes the few queries the kernel hands back (arena
// or row-cap overflow: the plain path; large results: the multi-CTA
// reorder).  Also the autotuner of the kernel's CTA shape.
#include <string.h>

#include <algorithm>
#include <vector>

#include "batch.cuh"
#include "join.cuh"
#include "plan.h"
#include "query.cuh"
#include "store.cuh"

struct gsmat_batch {
    const gsmat_store *S = nullptr;
    int n = 0;
    gsmat_batch_config cfg{};
    int grid = 0;
    std::vector<gs::BQuery> hq;
    std::vector<gs::BStep> hs;
    std::vector<std::vector<gsmat_pattern>> pats;
    std::vector<std::vector<int32_t>> plan_vars;
    gs::DevBuf prog, arena, ctrl, results_dev;
    std::vector<gs::DevBuf> seg_outs;  // columns of the results reordered together after the kernel
    gs::DevBuf compact;                // results copied out of the arena (compact_results)
    gs::BResult *results_host = nullptr;   // pinned
    unsigned long long *ctrl_host = nullptr;  // pinned: queue head | arena top
    cudaStream_t priv = nullptr;
    cudaEvent_t ev_in = nullptr, ev_a = nullptr, ev_b = nullptr, ev_done = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<gsmat_table *> owned;  // per query: plain-path or reordered table, else null
    std::vector<int32_t> path;         // 0 kernel, 1 plain path, 2 kernel + multi-CTA reorder
    std::vector<gs::BResult> results_final;  // descriptors after finish (ordinary host memory)
    bool borrowed = false;             // stream, events and pinned buffers belong to a server slot
    gsmat_batch_stats_t stats{};

    ~gsmat_batch() {
        for (auto *t : owned) delete t;
        owned.clear();
        if (borrowed) {
            prog.release();
            arena.release();
            ctrl.release();
            results_dev.release();
            seg_outs.clear();
            compact.release();
            return;
        }
        if (priv) cudaStreamSynchronize(priv);
        prog.release();
        arena.release();
        ctrl.release();
        results_dev.release();
        seg_outs.clear();
        compact.release();
        if (gexec) cudaGraphExecDestroy(gexec);
        if (results_host) cudaFreeHost(results_host);
        if (ctrl_host) cudaFreeHost(ctrl_host);
        for (cudaEvent_t e : {ev_in, ev_a, ev_b, ev_done}) {
            if (e) cudaEventDestroy(e);
        }
        if (priv) cudaStreamDestroy(priv);
    }
};

namespace gs {

int device_sm_count();

namespace {

gsmat_batch_config default_config() {
    gsmat_batch_config c;
    memset(&c, 0, sizeof(c));
    c.block = 256;
    c.ctas_per_sm = 4;
    c.arena_bytes = (int64_t)8 << 30;
    c.max_rows = (int64_t)1 << 22;
    c.use_graph = 1;
    c.expand_slots = 1;
    return c;
}

int resolve_config(const gsmat_batch_config *in, gsmat_batch_config *out) {
    gsmat_batch_config c = default_config();
    if (in) {
        if (in->block) c.block = in->block;
        if (in->ctas_per_sm) c.ctas_per_sm = in->ctas_per_sm;
        if (in->arena_bytes) c.arena_bytes = in->arena_bytes;
        if (in->max_rows) c.max_rows = in->max_rows;
        c.use_graph = in->use_graph;
        c.compact_results = in->compact_results;
        if (c.compact_results) c.use_graph = 0;  // the arena is re-allocated per run
        c.reorder_mode = in->reorder_mode;
        c.plan_cost = in->plan_cost;
        if (in->expand_slots) c.expand_slots = in->expand_slots;
    }
    if (c.expand_slots != 1 && c.expand_slots != 4) {
        return set_error(GSMAT_ERR_INVALID_ARG, "bad batch expand_slots %d (1 or 4)", c.expand_slots);
    }
    if (c.plan_cost != 0 && c.plan_cost != 1) {
        return set_error(GSMAT_ERR_INVALID_ARG, "bad batch plan_cost %d (0 or 1)", c.plan_cost);
    }
    if (c.reorder_mode < 0 || c.reorder_mode > (int)GSMAT_SORT_GATHER) {
        return set_error(GSMAT_ERR_INVALID_ARG, "bad batch reorder_mode %d", c.reorder_mode);
    }
    if (c.block != 128 && c.block != 256 && c.block != 512) {
        return set_error(GSMAT_ERR_INVALID_ARG, "batch block must be 128, 256 or 512 (got %d)", c.block);
    }
    if (c.ctas_per_sm < 1 || c.ctas_per_sm > 16 || c.arena_bytes < (1 << 20) || c.max_rows < 1 ||
        c.max_rows > INT32_MAX - 2) {
        return set_error(GSMAT_ERR_INVALID_ARG, "bad batch configuration");
    }
    *out = c;
    return GSMAT_OK;
}

// The kernel's arguments for the current buffers.
BatchArgs make_args(gsmat_batch *B) {
    BatchArgs a;
    a.sv = B->S->view;
    a.sides = B->S->pred_side_dev.as<PredSide>();
    a.n_pred = B->S->n_pred;
    a.bits = std::max(1, bits_for((uint64_t)std::max(B->S->max_entity, 0)));
    a.queries = B->prog.as<BQuery>();
    a.steps = reinterpret_cast<const BStep *>(B->prog.as<char>() + round_up(sizeof(BQuery) * B->n, 256));
    a.n_queries = B->n;
    a.results = B->results_dev.as<BResult>();
    a.arena = B->arena.as<char>();
    a.arena_cap = (unsigned long long)B->arena.bytes;
    a.queue_head = reinterpret_cast<unsigned int *>(B->ctrl.as<unsigned long long>());
    a.arena_top = B->ctrl.as<unsigned long long>() + 1;
    a.max_rows = B->cfg.max_rows;
    return a;
}

// Reset the queue and the arena, run the kernel, copy the descriptors back.
int enqueue_device_work(gsmat_batch *B) {
    GS_CUDA(cudaMemsetAsync(B->ctrl.p, 0, 2 * sizeof(unsigned long long), B->priv));
    BatchArgs a = make_args(B);
    GS_TRY(launch_batch_kernel(a, B->cfg.block, B->cfg.expand_slots, B->grid, B->priv));
    GS_CUDA(cudaMemcpyAsync(B->results_host, B->results_dev.p, sizeof(BResult) * B->n, cudaMemcpyDeviceToHost,
                            B->priv));
    GS_CUDA(cudaMemcpyAsync(B->ctrl_host, B->ctrl.p, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, B->priv));
    return GSMAT_OK;
}

int capture_graph(gsmat_batch *B) {
    if (B->gexec) {
        cudaGraphExecDestroy(B->gexec);
        B->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    GS_CUDA(cudaStreamBeginCapture(B->priv, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_device_work(B);
    cudaError_t e = cudaStreamEndCapture(B->priv, &g);
    if (rc != GSMAT_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return set_error(GSMAT_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&B->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        B->gexec = nullptr;
        return set_error(GSMAT_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return GSMAT_OK;
}

int prepare(const gsmat_store *S, const gsmat_bgp *bgps, int32_t n, const gsmat_batch_config *cfg_in,
            cudaStream_t user_st, const BatchResources *res, gsmat_batch *B) {
    if (!S || !bgps || n < 1) return set_error(GSMAT_ERR_INVALID_ARG, "store, bgps or n");
    B->S = S;
    B->n = n;
    GS_TRY(resolve_config(cfg_in, &B->cfg));
    B->grid = device_sm_count() * B->cfg.ctas_per_sm;
    if (res) {
        if (res->cap < n) return set_error(GSMAT_ERR_INVALID_ARG, "borrowed buffers hold %d results, not %d", res->cap, n);
        B->borrowed = true;
        B->priv = res->st;
        B->ev_in = res->ev[0];
        B->ev_a = res->ev[1];
        B->ev_b = res->ev[2];
        B->ev_done = res->ev[3];
        B->results_host = res->results_host;
        B->ctrl_host = res->ctrl_host;
    } else {
        GS_CUDA(cudaStreamCreateWithFlags(&B->priv, cudaStreamNonBlocking));
        for (cudaEvent_t *e : {&B->ev_in, &B->ev_a, &B->ev_b, &B->ev_done}) GS_CUDA(cudaEventCreate(e));
        GS_CUDA(cudaEventRecord(B->ev_in, user_st));
        GS_CUDA(cudaStreamWaitEvent(B->priv, B->ev_in, 0));
    }
    B->pats.resize(n);
    B->plan_vars.resize(n);
    for (int i = 0; i < n; ++i) {
        GS_TRY(validate_bgp(bgps[i].pats, bgps[i].n_pats, bgps[i].n_vars));
        B->pats[i].assign(bgps[i].pats, bgps[i].pats + bgps[i].n_pats);
    }
    // constant rows of every query, one lookup kernel
    std::vector<int32_t> req;
    std::vector<std::vector<int>> rs(n), ro(n);
    std::vector<std::vector<int32_t>> slot(n);
    std::vector<char> absent(n, 0);
    for (int i = 0; i < n; ++i) {
        const int np = bgps[i].n_pats;
        rs[i].assign(np, -1);
        ro[i].assign(np, -1);
        slot[i].assign(np, -1);
        for (int k = 0; k < np; ++k) {
            const gsmat_pattern &p = bgps[i].pats[k];
            slot[i][k] = S->slot_of(p.p);
            if (slot[i][k] < 0) {
                absent[i] = 1;
                continue;
            }
            if (!p.s_var) {
                rs[i][k] = (int)req.size() / 3;
                req.insert(req.end(), {slot[i][k], 0, p.s});
            }
            if (!p.o_var) {
                ro[i][k] = (int)req.size() / 3;
                req.insert(req.end(), {slot[i][k], 1, p.o});
            }
        }
    }
    const int n_req = (int)req.size() / 3;
    std::vector<int32_t> rng(2 * (size_t)n_req);
    if (n_req > 0) {
        DevBuf d;
        GS_TRY(d.alloc(sizeof(int32_t) * (req.size() + rng.size()), B->priv));
        GS_CUDA(cudaMemcpyAsync(d.p, req.data(), sizeof(int32_t) * req.size(), cudaMemcpyHostToDevice, B->priv));
        int32_t *d_out = d.as<int32_t>() + req.size();
        GS_TRY(launch_const_lookup(S->view, S->pred_side_dev.as<PredSide>(), S->n_pred, d.as<int32_t>(), n_req, d_out,
                                   B->priv));
        GS_CUDA(cudaMemcpyAsync(rng.data(), d_out, sizeof(int32_t) * rng.size(), cudaMemcpyDeviceToHost, B->priv));
        GS_CUDA(cudaStreamSynchronize(B->priv));
    }
    auto row_len = [&](int r) -> int64_t { return r < 0 ? 0 : (int64_t)rng[2 * r + 1] - rng[2 * r]; };
    // plans -> step programs
    B->hq.resize(n);
    for (int i = 0; i < n; ++i) {
        const int np = bgps[i].n_pats;
        const gsmat_pattern *P = bgps[i].pats;
        std::vector<int64_t> keys(np);
        std::vector<gsmat_pred_stats> st(np);
        for (int k = 0; k < np; ++k) {
            memset(&st[k], 0, sizeof(st[k]));
            const int sl = slot[i][k];
            if (sl < 0) {
                keys[k] = 0;
                continue;
            }
            st[k].nnz = S->side[0][sl].nnz;
            st[k].nr_s = S->side[0][sl].nrows;
            st[k].nr_o = S->side[1][sl].nrows;
            if (!P[k].s_var && !P[k].o_var) keys[k] = std::min(row_len(rs[i][k]), row_len(ro[i][k]));
            else if (!P[k].s_var) keys[k] = row_len(rs[i][k]);
            else if (!P[k].o_var) keys[k] = row_len(ro[i][k]);
            else keys[k] = st[k].nnz;
        }
        std::vector<int32_t> order(np), kinds(np);
        GS_TRY((B->cfg.plan_cost ? plan_bgp_cost : plan_bgp)(P, np, keys.data(), st.data(), order.data(),
                                                             kinds.data(), nullptr));
        BQuery &Q = B->hq[i];
        memset(&Q, 0, sizeof(Q));
        Q.step0 = (int32_t)B->hs.size();
        Q.n_steps = np;
        Q.n_vars = bgps[i].n_vars;
        Q.absent = absent[i];
        // intersect-expand fusion, as on the plain path: an EXPAND of a new
        // variable v from a bound variable and a later FILTER joining v with
        // a variable bound before the EXPAND (or a constant) run as one step
        std::vector<int> partner(np, -1);
        std::vector<char> fused(np, 0);
        {
            uint64_t bound = 0;
            for (int s = 0; s < np; ++s) {
                const gsmat_pattern &p = P[order[s]];
                const bool from_var = (kinds[s] == GSMAT_STEP_EXPAND_S && p.s_var) ||
                                      (kinds[s] == GSMAT_STEP_EXPAND_O && p.o_var);
                if (from_var && !fused[s]) {
                    const int32_t v = kinds[s] == GSMAT_STEP_EXPAND_S ? p.o : p.s;
                    for (int t = s + 1; t < np; ++t) {
                        if (kinds[t] != GSMAT_STEP_FILTER || fused[t]) continue;
                        const gsmat_pattern &f = P[order[t]];
                        if (f.s_var && f.o_var && f.s == f.o) continue;
                        const bool v_is_s = f.s_var && f.s == v;
                        const bool v_is_o = f.o_var && f.o == v;
                        if (v_is_s == v_is_o) continue;
                        const bool other_known = v_is_s ? (!f.o_var || ((bound >> f.o) & 1))
                                                        : (!f.s_var || ((bound >> f.s) & 1));
                        if (!other_known) continue;
                        partner[s] = t;
                        fused[t] = 1;
                        break;
                    }
                }
                if (p.s_var) bound |= uint64_t(1) << p.s;
                if (p.o_var) bound |= uint64_t(1) << p.o;
            }
        }
        int col_of_var[32];
        for (int v = 0; v < 32; ++v) col_of_var[v] = -1;
        int ncols = 0;
        std::vector<int32_t> &pv = B->plan_vars[i];
        for (int s = 0; s < np; ++s) {
            const int k = order[s];
            const gsmat_pattern &p = P[k];
            BStep S1;
            memset(&S1, 0, sizeof(S1));
            S1.kind = kinds[s];
            if (fused[s]) {
                S1.kind = GSMAT_STEP_FUSED;  // runs inside the INTERSECT before it
                B->hs.push_back(S1);
                continue;
            }
            if (partner[s] >= 0) {
                const gsmat_pattern &f = P[order[partner[s]]];
                const int32_t v = S1.kind == GSMAT_STEP_EXPAND_S ? p.o : p.s;
                const bool v_is_s = f.s_var && f.s == v;
                const bool b_var = v_is_s ? f.o_var : f.s_var;
                const int32_t b = v_is_s ? f.o : f.s;
                S1.a_side = S1.kind == GSMAT_STEP_EXPAND_S ? 0 : 1;
                S1.f_slot = slot[i][order[partner[s]]];
                S1.f_side = v_is_s ? 1 : 0;
                S1.b_col = b_var ? col_of_var[b] : -1;
                S1.b_const = b_var ? 0 : b;
            }
            S1.slot = slot[i][k] < 0 ? 0 : slot[i][k];
            S1.s_col = (p.s_var && col_of_var[p.s] >= 0) ? col_of_var[p.s] : -1;
            S1.o_col = (p.o_var && col_of_var[p.o] >= 0) ? col_of_var[p.o] : -1;
            S1.s_const = p.s_var ? 0 : p.s;
            S1.o_const = p.o_var ? 0 : p.o;
            if (S1.kind == GSMAT_STEP_EXPAND_S) {
                if (!p.s_var && rs[i][k] >= 0) {
                    S1.c_first = rng[2 * rs[i][k]];
                    S1.c_last = rng[2 * rs[i][k] + 1];
                }
                col_of_var[p.o] = ncols++;
                pv.push_back(p.o);
            } else if (S1.kind == GSMAT_STEP_EXPAND_O) {
                if (!p.o_var && ro[i][k] >= 0) {
                    S1.c_first = rng[2 * ro[i][k]];
                    S1.c_last = rng[2 * ro[i][k] + 1];
                }
                col_of_var[p.s] = ncols++;
                pv.push_back(p.s);
            } else if (S1.kind == GSMAT_STEP_CROSS) {
                S1.diag = p.s == p.o ? 1 : 0;
                S1.swap = (!S1.diag && p.o < p.s) ? 1 : 0;  // lower variable id first
                const int32_t first = S1.swap ? p.o : p.s, second = S1.swap ? p.s : p.o;
                col_of_var[first] = ncols++;
                pv.push_back(first);
                if (!S1.diag) {
                    col_of_var[second] = ncols++;
                    pv.push_back(second);
                }
            }
            if (partner[s] >= 0) S1.kind = GSMAT_STEP_INTERSECT;
            B->hs.push_back(S1);
        }
        for (int v = 0; v < Q.n_vars; ++v) Q.col_of_var[v] = col_of_var[v];
        Q.m_sort = leading_sort_vars(pv.data(), (int)pv.size());
    }
    // device buffers
    const size_t q_bytes = round_up(sizeof(BQuery) * n, 256);
    const size_t prog_bytes = q_bytes + sizeof(BStep) * std::max<size_t>(1, B->hs.size());
    GS_TRY(B->prog.alloc(prog_bytes, B->priv));
    GS_CUDA(cudaMemcpyAsync(B->prog.p, B->hq.data(), sizeof(BQuery) * n, cudaMemcpyHostToDevice, B->priv));
    if (!B->hs.empty()) {
        GS_CUDA(cudaMemcpyAsync(B->prog.as<char>() + q_bytes, B->hs.data(), sizeof(BStep) * B->hs.size(),
                                cudaMemcpyHostToDevice, B->priv));
    }
    GS_TRY(B->arena.alloc((size_t)B->cfg.arena_bytes, B->priv));
    GS_TRY(B->ctrl.alloc(2 * sizeof(unsigned long long), B->priv));
    GS_TRY(B->results_dev.alloc(sizeof(BResult) * n, B->priv));
    if (!B->borrowed) {
        GS_CUDA(cudaMallocHost((void **)&B->results_host, sizeof(BResult) * n));
        GS_CUDA(cudaMallocHost((void **)&B->ctrl_host, 2 * sizeof(unsigned long long)));
    }
    GS_CUDA(cudaStreamSynchronize(B->priv));
    for (DevBuf *d : {&B->prog, &B->arena, &B->ctrl, &B->results_dev}) d->st = nullptr;
    B->owned.assign(n, nullptr);
    B->path.assign(n, 0);
    if (B->cfg.use_graph) GS_TRY(capture_graph(B));
    return GSMAT_OK;
}

// The results the kernel left unsorted (more rows than its shared-memory
// sort) are reordered together, one group per number m of leading sort
// variables: a segmented least-significant-digit radix reorder whose last
// (most significant) key holds the result's index above its first
// variables, then one gather.
// The descriptors followed by the int64 array of their first rows (what the
// segmented kernels search), in one device buffer.
int upload_segs(const std::vector<SegDesc> &segs, DevBuf &d, cudaStream_t st) {
    const size_t n = segs.size();
    std::vector<char> h(sizeof(SegDesc) * n + sizeof(int64_t) * n);
    memcpy(h.data(), segs.data(), sizeof(SegDesc) * n);
    int64_t *start = reinterpret_cast<int64_t *>(h.data() + sizeof(SegDesc) * n);
    for (size_t k = 0; k < n; ++k) start[k] = segs[k].row_off;
    GS_TRY(d.alloc(h.size(), st));
    // a copy from pageable memory is staged before the call returns
    GS_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size(), cudaMemcpyHostToDevice, st));
    return GSMAT_OK;
}

int reorder_group(gsmat_batch *B, const std::vector<int> &qs, int m, int bits) {
    const int seg_bits = std::max(1, bits_for((uint64_t)(qs.size() - 1)));
    std::vector<SegDesc> segs;
    int64_t total = 0, out_words = 0;
    for (int i : qs) {
        const BResult &R = B->results_host[i];
        SegDesc d;
        memset(&d, 0, sizeof(d));
        d.row_off = total;
        d.rows = R.rows;
        d.m = m;
        d.V = R.ncols;
        for (int v = 0; v < R.ncols; ++v) d.col[v] = R.col[v];
        segs.push_back(d);
        total += R.rows;
        out_words += R.rows * R.ncols;
    }
    if (total > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "batch reorder of %lld rows", (long long)total);
    DevBuf out;
    GS_TRY(out.alloc(sizeof(int32_t) * (size_t)out_words, B->priv));
    int64_t w = 0;
    for (SegDesc &d : segs) {
        d.out = out.as<int32_t>() + w;
        w += d.rows * d.V;
    }
    DevBuf d_segs, keys, perm, err;
    GS_TRY(upload_segs(segs, d_segs, B->priv));
    GS_TRY(err.alloc(sizeof(int), B->priv));
    GS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), B->priv));
    // The other variables travel with the key when they fit 64 bits, the
    // key (with the segment index) one word of at most 40 bits, and the
    // rows are well beyond L2 (as the plain reorder decides): no gather.
    int max_rest = 0;
    for (const SegDesc &d : segs) max_rest = std::max(max_rest, d.V - m);
    const int kb_all = m * bits;
    const int key_bits_all = kb_all + seg_bits;
    const bool can_carry = kb_all + seg_bits <= 64 && max_rest > 0 && max_rest * bits <= 64;
    const int mode = B->cfg.reorder_mode;
    const bool carry = mode == GSMAT_SORT_CARRY ||
                       (mode == 0 && key_bits_all <= 40 && (double)total * max_rest * 4.0 > 256.0 * (1 << 20));
    if (can_carry && carry) {
        DevBuf pay;
        GS_TRY(keys.alloc(sizeof(uint64_t) * (size_t)total, B->priv));
        GS_TRY(pay.alloc(sizeof(uint64_t) * (size_t)total, B->priv));
        GS_TRY(launch_seg_pack_wide(d_segs.as<SegDesc>(), (int)segs.size(), bits, m, kb_all, total,
                                    keys.as<uint64_t>(), pay.as<uint64_t>(), B->priv));
        GS_TRY(radix_sort_u64_wide(keys.as<uint64_t>(), pay.as<uint64_t>(), total, 0, kb_all + seg_bits, B->priv,
                                   err.as<int>()));
        GS_TRY(launch_seg_unpack_wide(d_segs.as<SegDesc>(), (int)segs.size(), bits, m, total, keys.as<uint64_t>(),
                                      pay.as<uint64_t>(), B->priv));
    } else {
        GS_TRY(keys.alloc(sizeof(uint64_t) * (size_t)total, B->priv));
        GS_TRY(perm.alloc(sizeof(uint32_t) * (size_t)total, B->priv));
        // chunks: head [0, h) shares the key with the segment index; the tail
        // [h, m) in chunks of per_key variables, sorted first
        const int per_key = 64 / bits;
        const int h = std::min(m, (64 - seg_bits) / bits);
        std::vector<std::pair<int, int>> chunks;  // least significant first
        for (int e = m; e > h;) {
            const int b0 = std::max(h, e - per_key);
            chunks.push_back({b0, e});
            e = b0;
        }
        chunks.push_back({0, h});
        // a chunk whose key bits and the source position fit one 64-bit word
        // sorts keys alone (8 bytes per row and pass instead of 12)
        const int idx_bits = std::max(1, bits_for((uint64_t)(total - 1)));
        for (size_t c = 0; c < chunks.size(); ++c) {
            const int vb = chunks[c].first, ve = chunks[c].second;
            const bool last = c + 1 == chunks.size();
            const int kb = (ve - vb) * bits;
            const int key_bits = last ? kb + seg_bits : kb;
            const bool packed = key_bits + idx_bits <= 64;
            GS_TRY(launch_seg_pack(d_segs.as<SegDesc>(), (int)segs.size(), bits, vb, ve, last ? kb : -1,
                                   packed ? idx_bits : 0, c == 0 ? nullptr : perm.as<uint32_t>(), total,
                                   keys.as<uint64_t>(), perm.as<uint32_t>(), B->priv));
            if (packed) {
                GS_TRY(radix_sort_u64(keys.as<uint64_t>(), nullptr, total, idx_bits, idx_bits + key_bits, B->priv,
                                      err.as<int>()));
                GS_TRY(launch_key_low_bits(keys.as<uint64_t>(), idx_bits, total, perm.as<uint32_t>(), B->priv));
            } else {
                GS_TRY(radix_sort_u64(keys.as<uint64_t>(), perm.as<uint32_t>(), total, 0, key_bits, B->priv,
                                      err.as<int>()));
            }
        }
        GS_TRY(launch_seg_gather(d_segs.as<SegDesc>(), (int)segs.size(), total, perm.as<uint32_t>(), B->priv));
    }
    int herr = 0;
    GS_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, B->priv));
    GS_CUDA(cudaStreamSynchronize(B->priv));
    if (herr) return set_error(GSMAT_ERR_DEVICE_CHECK, "batch reorder: a bounded wait expired");
    for (size_t k = 0; k < segs.size(); ++k) {
        BResult &R = B->results_host[qs[k]];
        for (int v = 0; v < R.ncols; ++v) R.col[v] = segs[k].out + (size_t)v * segs[k].rows;
        R.status = BR_OK;
        B->path[qs[k]] = 2;
    }
    out.st = nullptr;
    B->seg_outs.push_back(std::move(out));
    return GSMAT_OK;
}

int reorder_large_results(gsmat_batch *B) {
    B->seg_outs.clear();
    std::vector<std::vector<int>> by_m(33);
    for (int i = 0; i < B->n; ++i) {
        B->path[i] = 0;
        if (B->results_host[i].status == BR_NEEDS_SORT) by_m[B->hq[i].m_sort].push_back(i);
    }
    const int bits = std::max(1, bits_for((uint64_t)std::max(B->S->max_entity, 0)));
    for (int m = 1; m <= 32; ++m) {
        if (!by_m[m].empty()) GS_TRY(reorder_group(B, by_m[m], m, bits));
    }
    return GSMAT_OK;
}

// Copy every kernel-path result into one right-sized buffer (one
// segmented copy kernel) and release the arena and reorder buffers.
int compact_results(gsmat_batch *B) {
    std::vector<SegDesc> segs;
    std::vector<int> qi;
    int64_t rows = 0, words = 0;
    for (int i = 0; i < B->n; ++i) {
        const BResult &R = B->results_host[i];
        if (B->owned[i] || R.status != BR_OK || R.rows == 0 || R.ncols == 0) continue;
        SegDesc d;
        memset(&d, 0, sizeof(d));
        d.row_off = rows;
        d.rows = R.rows;
        d.V = R.ncols;
        for (int v = 0; v < R.ncols; ++v) d.col[v] = R.col[v];
        segs.push_back(d);
        qi.push_back(i);
        rows += R.rows;
        words += R.rows * R.ncols;
    }
    B->compact.release();
    if (!segs.empty()) {
        GS_TRY(B->compact.alloc(sizeof(int32_t) * (size_t)words, B->priv));
        int64_t w = 0;
        for (SegDesc &d : segs) {
            d.out = B->compact.as<int32_t>() + w;
            w += d.rows * d.V;
        }
        DevBuf d_segs;
        GS_TRY(upload_segs(segs, d_segs, B->priv));
        GS_TRY(launch_seg_gather(d_segs.as<SegDesc>(), (int)segs.size(), rows, nullptr, B->priv));
        GS_CUDA(cudaStreamSynchronize(B->priv));
        for (size_t k = 0; k < segs.size(); ++k) {
            BResult &R = B->results_host[qi[k]];
            for (int v = 0; v < R.ncols; ++v) R.col[v] = segs[k].out + (size_t)v * segs[k].rows;
        }
        B->compact.st = nullptr;
    }
    // a result with no rows or columns keeps no pointer into the arena
    for (int i = 0; i < B->n; ++i) {
        BResult &R = B->results_host[i];
        if (!B->owned[i] && (R.rows == 0 || R.ncols == 0)) {
            for (int v = 0; v < 32; ++v) R.col[v] = nullptr;
        }
    }
    B->arena.release();
    B->seg_outs.clear();
    return GSMAT_OK;
}

// Device work only (no fallbacks); kernel time in *ms.
int run_device(gsmat_batch *B, float *ms) {
    GS_CUDA(cudaEventRecord(B->ev_a, B->priv));
    if (B->gexec) {
        GS_CUDA(cudaGraphLaunch(B->gexec, B->priv));
    } else {
        GS_TRY(enqueue_device_work(B));
    }
    GS_CUDA(cudaEventRecord(B->ev_b, B->priv));
    GS_CUDA(cudaStreamSynchronize(B->priv));
    GS_CUDA(cudaEventElapsedTime(ms, B->ev_a, B->ev_b));
    return GSMAT_OK;
}

// Enqueue the device work of a run on the batch's stream and return.
int launch_async(gsmat_batch *B) {
    for (auto *&t : B->owned) {
        delete t;
        t = nullptr;
    }
    if (!B->arena.p) {  // released by the previous run's compaction
        GS_TRY(B->arena.alloc((size_t)B->cfg.arena_bytes, B->priv));
        B->arena.st = nullptr;
    }
    GS_CUDA(cudaEventRecord(B->ev_a, B->priv));
    if (B->gexec) {
        GS_CUDA(cudaGraphLaunch(B->gexec, B->priv));
    } else {
        GS_TRY(enqueue_device_work(B));
    }
    GS_CUDA(cudaEventRecord(B->ev_b, B->priv));
    return GSMAT_OK;
}

// Wait for the run's device work, then finish the results the kernel handed
// back (batched reorder of large results, plain-path re-runs).
int finish(gsmat_batch *B) {
    GS_CUDA(cudaEventSynchronize(B->ev_b));
    float ms = 0;
    GS_CUDA(cudaEventElapsedTime(&ms, B->ev_a, B->ev_b));
    gsmat_batch_stats_t &s = B->stats;
    memset(&s, 0, sizeof(s));
    s.n_queries = B->n;
    s.kernel_ms = ms;
    s.arena_used = (int64_t)std::min<unsigned long long>(B->ctrl_host[1], (unsigned long long)B->arena.bytes);
    s.block = B->cfg.block;
    s.grid = B->grid;
    for (const BStep &st : B->hs) s.n_intersect += st.kind == GSMAT_STEP_INTERSECT ? 1 : 0;
    GS_CUDA(cudaEventRecord(B->ev_a, B->priv));
    GS_TRY(reorder_large_results(B));
    GS_CUDA(cudaEventRecord(B->ev_b, B->priv));
    GS_CUDA(cudaEventSynchronize(B->ev_b));
    float rms = 0;
    GS_CUDA(cudaEventElapsedTime(&rms, B->ev_a, B->ev_b));
    s.reorder_ms = rms;
    for (int i = 0; i < B->n; ++i) {
        const BResult &R = B->results_host[i];
        if (B->path[i] == 2 && R.status == BR_OK) {
            s.n_reordered++;
        } else if (R.status == BR_OK) {
            B->path[i] = 0;
            s.n_in_kernel++;
        } else if (R.status == BR_NEEDS_SORT) {
            const std::vector<int32_t> &pv = B->plan_vars[i];
            const int V = (int)pv.size();
            std::vector<const int32_t *> cols(V);
            for (int c = 0; c < V; ++c) cols[c] = R.col[pv[c]];
            GS_TRY(reorder_view(B->S, cols.data(), pv.data(), V, R.rows, B->priv, &B->owned[i]));
            B->path[i] = 2;
            s.n_reordered++;
        } else {
            GS_TRY(query_run(B->S, B->pats[i].data(), (int)B->pats[i].size(), B->hq[i].n_vars,
                             B->cfg.plan_cost ? GSMAT_PLAN_COST : GSMAT_SORTED, B->priv,
                             &B->owned[i]));
            B->path[i] = 1;
            s.n_fallback++;
        }
    }
    if (B->cfg.compact_results) GS_TRY(compact_results(B));
    B->results_final.assign(B->results_host, B->results_host + B->n);
    return GSMAT_OK;
}

int execute(gsmat_batch *B, cudaStream_t user_st) {
    GS_CUDA(cudaEventRecord(B->ev_in, user_st));
    GS_CUDA(cudaStreamWaitEvent(B->priv, B->ev_in, 0));
    KernelTimer timer("batch_kernel", B->priv, 0.0, (double)B->n);
    GS_TRY(launch_async(B));
    timer.stop();
    GS_TRY(finish(B));
    GS_CUDA(cudaEventRecord(B->ev_done, B->priv));
    GS_CUDA(cudaStreamWaitEvent(user_st, B->ev_done, 0));
    profile_flush();
    return GSMAT_OK;
}

// Column c (variable order) of query i and its row count.
int result_view(const gsmat_batch *B, int32_t i, int64_t *rows, int32_t *cols, const int32_t **col_ptrs) {
    if (!B || i < 0 || i >= B->n) return set_error(GSMAT_ERR_INVALID_ARG, "bad batch or index");
    if (B->owned[i]) {
        const gsmat_table *T = B->owned[i];
        if (rows) *rows = T->rows;
        if (cols) *cols = T->ncols;
        if (col_ptrs) for (int c = 0; c < T->ncols; ++c) col_ptrs[c] = T->col[c];
        return GSMAT_OK;
    }
    if ((int)B->results_final.size() != B->n) return set_error(GSMAT_ERR_INVALID_ARG, "batch has not been executed");
    const BResult &R = B->results_final[i];
    if (rows) *rows = R.rows;
    if (cols) *cols = R.ncols;
    if (col_ptrs) for (int c = 0; c < R.ncols; ++c) col_ptrs[c] = R.col[c];
    return GSMAT_OK;
}

}  // namespace

int batch_prepare_with(const gsmat_store *S, const gsmat_bgp *bgps, int32_t n, const gsmat_batch_config *cfg,
                       cudaStream_t st, const BatchResources *res, gsmat_batch **out) {
    if (!out) return set_error(GSMAT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    gsmat_batch *B = new gsmat_batch();
    int rc = prepare(S, bgps, n, cfg, st, res, B);
    if (rc != GSMAT_OK) {
        delete B;
        return rc;
    }
    *out = B;
    return GSMAT_OK;
}

int batch_prepare(const gsmat_store *S, const gsmat_bgp *bgps, int32_t n, const gsmat_batch_config *cfg,
                  cudaStream_t st, gsmat_batch **out) {
    return batch_prepare_with(S, bgps, n, cfg, st, nullptr, out);
}

int batch_launch_async(gsmat_batch *B) { return launch_async(B); }
int batch_kernel_done(gsmat_batch *B) {
    const cudaError_t e = cudaEventQuery(B->ev_b);
    if (e == cudaErrorNotReady) return 0;
    if (e != cudaSuccess) cudaGetLastError();
    return 1;  // done, or failed: finish() reports the error
}
int batch_finish(gsmat_batch *B) { return finish(B); }
int batch_result_view(const gsmat_batch *B, int32_t i, int64_t *rows, int32_t *cols, const int32_t **col_ptrs) {
    return result_view(B, i, rows, cols, col_ptrs);
}

int batch_execute(gsmat_batch *B, cudaStream_t st) {
    if (!B) return set_error(GSMAT_ERR_INVALID_ARG, "batch is NULL");
    return execute(B, st);
}

int batch_result(const gsmat_batch *B, int32_t i, int64_t *rows, int32_t *cols, int32_t *path) {
    GS_TRY(result_view(B, i, rows, cols, nullptr));
    if (path) *path = B->path[i];
    return GSMAT_OK;
}

int batch_column(const gsmat_batch *B, int32_t i, int32_t c, const int32_t **d_col) {
    int32_t cols = 0;
    const int32_t *ptrs[32];
    GS_TRY(result_view(B, i, nullptr, &cols, ptrs));
    if (c < 0 || c >= cols || !d_col) return set_error(GSMAT_ERR_INVALID_ARG, "bad column");
    *d_col = ptrs[c];
    return GSMAT_OK;
}

int batch_copy(const gsmat_batch *B, int32_t i, int32_t *dst, int dst_on_device, cudaStream_t st) {
    int64_t rows = 0;
    int32_t cols = 0;
    const int32_t *ptrs[32];
    GS_TRY(result_view(B, i, &rows, &cols, ptrs));
    if (rows == 0 || cols == 0) return GSMAT_OK;
    if (!dst) return set_error(GSMAT_ERR_INVALID_ARG, "dst is NULL");
    Cols in;
    for (int c = 0; c < kMaxCols; ++c) in.c[c] = c < cols ? ptrs[c] : nullptr;
    if (dst_on_device) {
        GS_TRY(launch_interleave(in, cols, rows, dst, st));
        GS_CUDA(cudaStreamSynchronize(st));
        return GSMAT_OK;
    }
    DevBuf tmp;
    GS_TRY(tmp.alloc(sizeof(int32_t) * (size_t)rows * cols, st));
    GS_TRY(launch_interleave(in, cols, rows, tmp.as<int32_t>(), st));
    GS_CUDA(cudaMemcpyAsync(dst, tmp.p, sizeof(int32_t) * (size_t)rows * cols, cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    return GSMAT_OK;
}

void batch_free(gsmat_batch *B) { delete B; }

int batch_stats(const gsmat_batch *B, gsmat_batch_stats_t *s) {
    if (!B || !s) return set_error(GSMAT_ERR_INVALID_ARG, "NULL argument");
    *s = B->stats;
    return GSMAT_OK;
}

int batch_autotune(const gsmat_store *S, const gsmat_bgp *bgps, int32_t n, const gsmat_batch_config *base,
                   cudaStream_t st, gsmat_batch_config *best) {
    if (!best) return set_error(GSMAT_ERR_INVALID_ARG, "best is NULL");
    gsmat_batch_config cfg;
    GS_TRY(resolve_config(base, &cfg));
    cfg.use_graph = 0;
    gsmat_batch *B = nullptr;
    GS_TRY(batch_prepare(S, bgps, n, &cfg, st, &B));
    const int blocks[3] = {128, 256, 512};
    const int per_sm[4] = {1, 2, 4, 8};
    const int slots[2] = {1, 4};
    float best_ms = 3.4e38f;
    gsmat_batch_config pick = cfg;
    int rc = GSMAT_OK;
    for (int b : blocks) {
        for (int c : per_sm) {
            if (b * c > 2048) continue;  // threads per SM
            for (int e : slots) {
                B->cfg.block = b;
                B->cfg.ctas_per_sm = c;
                B->cfg.expand_slots = e;
                B->grid = device_sm_count() * c;
                float t_min = 3.4e38f;
                for (int rep = 0; rep < 3 && rc == GSMAT_OK; ++rep) {
                    float ms = 0;
                    rc = run_device(B, &ms);
                    if (rc == GSMAT_OK && rep > 0) t_min = std::min(t_min, ms);
                }
                if (rc != GSMAT_OK) break;
                if (t_min < best_ms) {
                    best_ms = t_min;
                    pick.block = b;
                    pick.ctas_per_sm = c;
                    pick.expand_slots = e;
                }
            }
            if (rc != GSMAT_OK) break;
        }
        if (rc != GSMAT_OK) break;
    }
    delete B;
    if (rc != GSMAT_OK) return rc;
    pick.use_graph = base ? base->use_graph : 1;
    *best = pick;
    return GSMAT_OK;
}

}  // namespace gs
