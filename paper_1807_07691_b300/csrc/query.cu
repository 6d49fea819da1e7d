// Query executor: Alg. 2 ("Query Execution", Sec. 6.3) over the plan of
// Alg. 1, one SM-based join (Alg. 3) per step, all on one stream.
//
// The running relation starts as the relation with one empty assignment;
// each plan step joins it with the next pattern's matrix:
//   FILTER   both ends known      -> membership filter + compaction
//   EXPAND   one end known        -> count + scan (Alg. 4), gather-expand
//            (from a constant: a Cartesian product with that row)
//   CROSS    no end known         -> Cartesian product with M_p (or with its
//                                    diagonal for ?x p ?x)
// A step whose input is the one-row, zero-column start relation returns the
// pattern's relation itself, as a view of the store (no copy).  Results are
// kept in plan column order, ascending (expansion preserves parent order and
// every row's entries are sorted), and reordered to variable order at the
// end by a stable radix sort on the few leading variables that need it.
#include <string.h>

#include <algorithm>
#include <vector>

#include "join.cuh"
#include "plan.h"
#include "query.cuh"
#include "select.cuh"
#include "store.cuh"

namespace gs {

int leading_sort_vars(const int32_t *plan_vars, int V) {
    for (int cand = 0; cand <= V; ++cand) {
        int want = cand;
        bool ok = true;
        for (int c = 0; c < V && ok; ++c) {
            if (plan_vars[c] < cand) continue;
            if (plan_vars[c] != want) ok = false;
            want++;
        }
        if (ok) return cand;
    }
    return V;
}

namespace {

struct Tbl {
    int64_t rows = 0;
    int ncols = 0;
    int32_t vars[kMaxCols];
    const int32_t *col[kMaxCols];
    DevBuf buf;  // owning storage; empty when the columns are a view of the store

    Cols cols() const {
        Cols c;
        for (int i = 0; i < kMaxCols; ++i) c.c[i] = i < ncols ? col[i] : nullptr;
        return c;
    }
    int col_of(int32_t var) const {
        for (int i = 0; i < ncols; ++i) if (vars[i] == var) return i;
        return -1;
    }
};

// Allocate ncols columns of `rows` rows (each 256-byte aligned).
int alloc_cols(Tbl &t, int ncols, int64_t rows, cudaStream_t st, OutCols *out) {
    const size_t stride = round_up((size_t)(rows > 0 ? rows : 1), 64);
    GS_TRY(t.buf.alloc(sizeof(int32_t) * stride * (size_t)(ncols > 0 ? ncols : 1), st));
    t.ncols = ncols;
    t.rows = rows;
    for (int c = 0; c < kMaxCols; ++c) {
        int32_t *p = c < ncols ? t.buf.as<int32_t>() + stride * c : nullptr;
        if (out) out->c[c] = p;
        if (c < ncols) t.col[c] = p;
    }
    return GSMAT_OK;
}

struct Ctx {
    const gsmat_store *S;
    cudaStream_t st;
    DevBuf qstat;  // [0] count / total, [1] error word (int)
    int64_t *h = nullptr;

    int64_t *d_count() { return qstat.as<int64_t>(); }
    int *d_err() { return reinterpret_cast<int *>(qstat.as<int64_t>() + 1); }

    // Read the count word and the error word; synchronises the stream.
    int read_count(int64_t *count) {
        GS_TRY(read_words(qstat.p, h, 2, st));
        if (*reinterpret_cast<int *>(h + 1)) return set_error(GSMAT_ERR_DEVICE_CHECK, "a bounded wait expired");
        *count = h[0];
        return GSMAT_OK;
    }
};

// Stable reorder of rows by the first m variables (variable order), then
// columns in variable order.  Input rows ascend in plan column order.
int canonical_order(Ctx &cx, Tbl &t, Tbl &out) {
    const int V = t.ncols;
    int32_t colof[kMaxCols];
    for (int v = 0; v < V; ++v) colof[v] = t.col_of(v);
    // smallest m: dropping variables 0..m-1 from the column order leaves
    // m, m+1, ..., V-1 in order (stable sort by a key over an input sorted
    // by S yields order (key, S))
    const int m = leading_sort_vars(t.vars, V);
    out.rows = t.rows;
    out.ncols = V;
    if (t.rows <= 1 || m == 0) {
        // only the column order changes
        for (int v = 0; v < V; ++v) {
            out.vars[v] = v;
            out.col[v] = t.col[colof[v]];
        }
        out.buf = std::move(t.buf);
        return GSMAT_OK;
    }
    const int bits = std::max(1, bits_for((uint64_t)std::max(cx.S->max_entity, 0)));
    Cols in;
    for (int v = 0; v < kMaxCols; ++v) in.c[v] = v < V ? t.col[colof[v]] : nullptr;
    OutCols oc;
    GS_TRY(alloc_cols(out, V, t.rows, cx.st, &oc));
    for (int v = 0; v < V; ++v) out.vars[v] = v;
    return reorder_rows(in, V, m, bits, t.rows, oc, cx.st, cx.d_err());
}

int run(const gsmat_store *S, const gsmat_pattern *pats, int n_pats, int n_vars, uint32_t flags, cudaStream_t st,
        gsmat_table *T, int shard, int n_shards) {
    GS_TRY(validate_bgp(pats, n_pats, n_vars));
    if (flags & ~(GSMAT_PLAN_ORDER | GSMAT_COUNT_ONLY | GSMAT_NO_INTERSECT | GSMAT_PLAN_COST)) {
        return set_error(GSMAT_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
    }
    T->id_bits = std::max(1, bits_for((uint64_t)std::max(S->max_entity, 0)));
    Ctx cx;
    cx.S = S;
    cx.st = st;
    cx.h = pinned_scratch(4 + 8 * GSMAT_MAX_PATTERNS);
    if (!cx.h) return set_error(GSMAT_ERR_CUDA, "pinned host scratch");
    GS_TRY(cx.qstat.alloc(4 * sizeof(int64_t), st));
    GS_CUDA(cudaMemsetAsync(cx.qstat.p, 0, 4 * sizeof(int64_t), st));

    // predicate slots, statistics and constant rows
    std::vector<int32_t> slot(n_pats);
    std::vector<gsmat_pred_stats> stats(n_pats);
    std::vector<int64_t> keys(n_pats);
    std::vector<int> req_s(n_pats, -1), req_o(n_pats, -1);
    std::vector<int32_t> req;
    bool absent = false;
    for (int i = 0; i < n_pats; ++i) {
        slot[i] = S->slot_of(pats[i].p);
        memset(&stats[i], 0, sizeof(stats[i]));
        stats[i].pred_id = pats[i].p;
        if (slot[i] < 0) {
            absent = true;
            continue;
        }
        stats[i].nnz = S->side[0][slot[i]].nnz;
        stats[i].nr_s = S->side[0][slot[i]].nrows;
        stats[i].nr_o = S->side[1][slot[i]].nrows;
        if (!pats[i].s_var) {
            req_s[i] = (int)req.size() / 3;
            req.insert(req.end(), {slot[i], 0, pats[i].s});
        }
        if (!pats[i].o_var) {
            req_o[i] = (int)req.size() / 3;
            req.insert(req.end(), {slot[i], 1, pats[i].o});
        }
    }
    const int n_req = (int)req.size() / 3;
    std::vector<int32_t> rng(2 * (size_t)n_req);
    if (n_req > 0 && !absent) {
        // requests and row ranges pass through the mapped scratch: the
        // kernel reads and writes it directly, no copy engine involved
        int32_t *hreq = reinterpret_cast<int32_t *>(cx.h + 4);
        int32_t *hout = hreq + req.size();
        memcpy(hreq, req.data(), sizeof(int32_t) * req.size());
        GS_TRY(launch_const_lookup(S->view, S->pred_side_dev.as<PredSide>(), S->n_pred,
                                   static_cast<const int32_t *>(pinned_scratch_device(hreq)), n_req,
                                   static_cast<int32_t *>(pinned_scratch_device(hout)), st));
        GS_TRY(wait_stream(st));
        memcpy(rng.data(), hout, sizeof(int32_t) * rng.size());
    }
    auto row_len = [&](int r) -> int64_t { return r < 0 ? 0 : (int64_t)rng[2 * r + 1] - rng[2 * r]; };
    for (int i = 0; i < n_pats; ++i) {
        if (slot[i] < 0) {
            keys[i] = 0;
        } else if (!pats[i].s_var && !pats[i].o_var) {
            keys[i] = std::min(row_len(req_s[i]), row_len(req_o[i]));
        } else if (!pats[i].s_var) {
            keys[i] = row_len(req_s[i]);
        } else if (!pats[i].o_var) {
            keys[i] = row_len(req_o[i]);
        } else {
            keys[i] = stats[i].nnz;
        }
    }
    gsmat_query_stats &qs = T->stats;
    memset(&qs, 0, sizeof(qs));
    qs.n_steps = n_pats;
    GS_TRY(((flags & GSMAT_PLAN_COST) ? plan_bgp_cost : plan_bgp)(pats, n_pats, keys.data(), stats.data(), qs.order,
                                                                   qs.kind, qs.est_rows));
    for (int s = 0; s < n_pats; ++s) {
        qs.est_cost += qs.est_rows[s];
        qs.rows[s] = -1;
    }
    // Constant rows first: when every pattern with one constant end and one
    // new variable can run first (its row depends on nothing) and every
    // other pattern then expands a variable those rows bind, the result is
    // the product of the constant rows (in variable order) joined with a
    // product per row of the expansions -- two product steps, no final
    // reorder.  Taken only when the constant rows' product (its size is
    // exact: the rows are known) stays within twice the estimated result and
    // 2^27 rows, so no intermediate appears that Alg. 1's order would keep
    // small.  Off for GSMAT_NO_INTERSECT, GSMAT_PLAN_ORDER and row shards.
    int fixed_prefix = 0;
    if (!(flags & (GSMAT_NO_INTERSECT | GSMAT_PLAN_ORDER)) && !absent && n_shards == 1 && n_pats >= 3) {
        std::vector<int32_t> fx, rest;
        uint64_t fvars = 0;
        bool ok = true;
        double prefix_rows = 1.0;
        for (int s = 0; s < n_pats && ok; ++s) {
            const int i = qs.order[s];
            const gsmat_pattern &p = pats[i];
            if (p.s_var != p.o_var) {  // one constant end, one variable
                const int32_t v = p.s_var ? p.s : p.o;
                if ((fvars >> v) & 1) ok = false;  // a second constant row for the same variable
                fvars |= uint64_t(1) << v;
                fx.push_back(i);
                prefix_rows *= (double)keys[i];
            } else {
                rest.push_back(i);
            }
        }
        double final_rows = prefix_rows;
        uint64_t bound = fvars;
        for (int32_t i : rest) {
            if (!ok) break;
            const gsmat_pattern &p = pats[i];
            const int kind = step_kind(p, bound);
            const bool from_prefix = (kind == GSMAT_STEP_EXPAND_S && p.s_var && ((fvars >> p.s) & 1)) ||
                                     (kind == GSMAT_STEP_EXPAND_O && p.o_var && ((fvars >> p.o) & 1));
            if (!from_prefix) {
                ok = false;
                break;
            }
            const double nr = kind == GSMAT_STEP_EXPAND_S ? (double)stats[i].nr_s : (double)stats[i].nr_o;
            final_rows *= nr > 0 ? (double)stats[i].nnz / nr : 0.0;
            bound |= uint64_t(1) << (kind == GSMAT_STEP_EXPAND_S ? p.o : p.s);
        }
        if (ok && fx.size() >= 2 && fx.size() <= (size_t)kMaxProdFactors && !rest.empty() && prefix_rows <= 2.0 * final_rows &&
            prefix_rows <= (double)(int64_t(1) << 27)) {
            uint64_t bnd = 0;
            double est = 1.0;
            int s = 0;
            for (const std::vector<int32_t> *part : {&fx, &rest}) {
                for (int32_t i : *part) {
                    const gsmat_pattern &p = pats[i];
                    const int kind = step_kind(p, bnd);
                    qs.order[s] = i;
                    qs.kind[s] = kind;
                    if (part == &fx) {
                        est *= (double)keys[i];
                    } else {
                        const double nr = kind == GSMAT_STEP_EXPAND_S ? (double)stats[i].nr_s : (double)stats[i].nr_o;
                        est *= nr > 0 ? (double)stats[i].nnz / nr : 0.0;
                    }
                    qs.est_rows[s] = est;
                    if (p.s_var) bnd |= uint64_t(1) << p.s;
                    if (p.o_var) bnd |= uint64_t(1) << p.o;
                    ++s;
                }
            }
            qs.est_cost = 0;
            for (int k = 0; k < n_pats; ++k) qs.est_cost += qs.est_rows[k];
            fixed_prefix = (int)fx.size();
        }
    }

    // variables in the order the plan binds them
    std::vector<int32_t> plan_vars;
    {
        uint64_t seen = 0;
        for (int s = 0; s < n_pats; ++s) {
            const gsmat_pattern &p = pats[qs.order[s]];
            // a CROSS of two new variables binds the lower id first (see the step)
            const bool swap = qs.kind[s] == GSMAT_STEP_CROSS && p.s_var && p.o_var && p.o < p.s;
            const int32_t a = swap ? p.o : p.s, b = swap ? p.s : p.o;
            const bool a_var = swap ? p.o_var : p.s_var, b_var = swap ? p.s_var : p.o_var;
            if (a_var && !((seen >> a) & 1)) { plan_vars.push_back(a); seen |= uint64_t(1) << a; }
            if (b_var && !((seen >> b) & 1)) { plan_vars.push_back(b); seen |= uint64_t(1) << b; }
        }
    }

    // Intersect-expand fusion: an EXPAND of a new variable v from a bound
    // variable, and a later FILTER whose pattern joins v with a variable
    // bound before the EXPAND (or a constant), run as one step whose new
    // column is the intersection of the two rows.  Applying the filter
    // early changes neither the rows nor their order.
    std::vector<int> partner(n_pats, -1);
    std::vector<char> fused(n_pats, 0);
    if (!(flags & GSMAT_NO_INTERSECT)) {
        uint64_t bound = 0;
        for (int s = 0; s < n_pats; ++s) {
            const gsmat_pattern &p = pats[qs.order[s]];
            const int kind = qs.kind[s];
            const bool from_var = (kind == GSMAT_STEP_EXPAND_S && p.s_var) || (kind == GSMAT_STEP_EXPAND_O && p.o_var);
            if (from_var && !fused[s]) {
                const int32_t v = kind == GSMAT_STEP_EXPAND_S ? p.o : p.s;
                for (int t = s + 1; t < n_pats; ++t) {
                    if (qs.kind[t] != GSMAT_STEP_FILTER || fused[t]) continue;
                    const gsmat_pattern &f = pats[qs.order[t]];
                    if (f.s_var && f.o_var && f.s == f.o) continue;
                    const bool v_is_s = f.s_var && f.s == v;
                    const bool v_is_o = f.o_var && f.o == v;
                    if (v_is_s == v_is_o) continue;
                    const bool other_known = v_is_s ? (!f.o_var || ((bound >> f.o) & 1)) : (!f.s_var || ((bound >> f.s) & 1));
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

    // Product of independent expansions: the longest suffix of the plan
    // whose steps each take their list from the table before the suffix or
    // from the store alone (EXPAND from a variable bound before it, EXPAND
    // from a constant, CROSS) runs as one product step (launch_product),
    // nested by variable id so that the result needs little or no final
    // reorder.  Off for GSMAT_NO_INTERSECT (one pattern per step) and for
    // GSMAT_PLAN_ORDER (the paper's binding order).
    int tail = n_pats;
    if (!(flags & (GSMAT_NO_INTERSECT | GSMAT_PLAN_ORDER)) && !absent) {
        std::vector<uint64_t> before(n_pats + 1, 0);  // variables bound by the steps before s
        for (int s = 0; s < n_pats; ++s) {
            const gsmat_pattern &p = pats[qs.order[s]];
            before[s + 1] = before[s] | (p.s_var ? uint64_t(1) << p.s : 0) | (p.o_var ? uint64_t(1) << p.o : 0);
        }
        auto independent = [&](int s, uint64_t pre) {
            if (fused[s] || partner[s] >= 0) return false;
            const gsmat_pattern &p = pats[qs.order[s]];
            switch (qs.kind[s]) {
                case GSMAT_STEP_EXPAND_S: return !p.s_var || ((pre >> p.s) & 1) != 0;
                case GSMAT_STEP_EXPAND_O: return !p.o_var || ((pre >> p.o) & 1) != 0;
                case GSMAT_STEP_CROSS: return p.s_var && p.o_var && p.s != p.o;
                default: return false;
            }
        };
        for (int t = n_pats - 1; t >= 0; --t) {
            bool ok = true;
            for (int s = t; s < n_pats && ok; ++s) ok = independent(s, before[t]);
            if (!ok) break;
            tail = t;
        }
        if (n_shards > 1 && tail == 0) tail = 1;  // shards split the first step's relation
        if (n_pats - tail > kMaxProdFactors) tail = n_pats - kMaxProdFactors;
        if (n_pats - tail < 2) tail = n_pats;
        if (fixed_prefix > 0) {
            // the constant rows run as one product; the rest (expansions of
            // their variables) as the tail, or step by step if it is one step
            tail = (n_pats - fixed_prefix >= 2 && n_pats - fixed_prefix <= kMaxProdFactors) ? fixed_prefix : n_pats;
        }
    }

    Tbl cur;
    cur.rows = absent ? 0 : 1;  // one empty assignment
    cur.ncols = 0;
    const bool count_only = (flags & GSMAT_COUNT_ONLY) != 0;
    // Steps [a, b) as one product step on `cur` (see launch_product);
    // count_rows: only the row count is needed (the query's last step).
    auto product_segment = [&](int a, int b, bool count_rows) -> int {
        struct Fac {
            int32_t v0, v1;  // the factor's variables (v1 = -1 for one)
            ProdFactor f;
        };
        std::vector<Fac> facs;
        for (int s = a; s < b; ++s) {
            const gsmat_pattern &p = pats[qs.order[s]];
            const int sl = slot[qs.order[s]];
            Fac x;
            memset(&x, 0, sizeof(x));
            x.v1 = -1;
            if (qs.kind[s] == GSMAT_STEP_CROSS) {
                // M_p from the side that puts the lower variable first, as a CROSS step does
                const int sd = p.o < p.s ? 1 : 0;
                const PredSide &pss = S->side[sd][sl];
                x.f.kind = kProdPairs;
                x.f.a = S->view.side[sd].key + pss.ent_base;
                x.f.b = S->view.side[sd].val + pss.ent_base;
                x.f.len = (uint32_t)pss.nnz;
                x.v0 = sd == 0 ? p.s : p.o;
                x.v1 = sd == 0 ? p.o : p.s;
            } else {
                const int side = qs.kind[s] == GSMAT_STEP_EXPAND_S ? 0 : 1;
                x.v0 = side == 0 ? p.o : p.s;
                if (side == 0 ? p.s_var : p.o_var) {
                    x.f.kind = kProdRow;
                    x.f.side = side;
                    x.f.xcol = cur.col_of(side == 0 ? p.s : p.o);
                    x.f.ps = S->side[side][sl];
                } else {
                    const int r = side == 0 ? req_s[qs.order[s]] : req_o[qs.order[s]];
                    x.f.kind = kProdList;
                    x.f.a = S->view.side[side].val + rng[2 * r];
                    x.f.len = (uint32_t)row_len(r);
                }
            }
            facs.push_back(x);
        }
        // outermost factor = smallest variable: inside every input row the
        // product's rows then ascend in variable order
        std::stable_sort(facs.begin(), facs.end(), [](const Fac &a, const Fac &b) { return a.v0 < b.v0; });
        ProdSpec spec;
        memset(&spec, 0, sizeof(spec));
        spec.nf = (int)facs.size();
        Tbl nxt;
        int col = cur.ncols;
        for (int c = 0; c < cur.ncols; ++c) nxt.vars[c] = cur.vars[c];
        uint64_t fixed = 1;  // product of the fixed factors' lengths, saturating
        const uint64_t kSat = uint64_t(1) << 40;
        for (int i = 0; i < spec.nf; ++i) {
            ProdFactor &f = spec.f[i];
            f = facs[i].f;
            f.out0 = col;
            nxt.vars[col++] = facs[i].v0;
            if (f.kind == kProdPairs) nxt.vars[col++] = facs[i].v1;
            if (f.kind == kProdRow) {
                f.slot = spec.nrow++;
            } else {
                f.div = make_fastdiv(f.len);
                fixed = (f.len != 0 && fixed > kSat / f.len) ? kSat : fixed * f.len;
            }
        }
        int64_t total = 0;
        const bool unit = cur.rows == 1 && cur.ncols == 0;
        if (unit) {
            // fixed lists only (a row factor needs a column of the table)
            total = (int64_t)fixed;
            if (total > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "product of %lld rows", (long long)total);
            if (!count_rows && total > 0) {
                OutCols oc;
                GS_TRY(alloc_cols(nxt, col, total, st, &oc));
                GS_TRY(launch_product_fixed(spec, total, oc, st));
            }
            // the plan-order intermediates are known exactly: running products
            uint64_t run_rows = 1;
            for (int s = a; s < b; ++s) {
                const gsmat_pattern &p = pats[qs.order[s]];
                const int sl = slot[qs.order[s]];
                uint64_t l;
                if (qs.kind[s] == GSMAT_STEP_CROSS) {
                    l = (uint64_t)S->side[p.o < p.s ? 1 : 0][sl].nnz;
                } else {
                    const bool sd0 = qs.kind[s] == GSMAT_STEP_EXPAND_S;
                    l = (uint64_t)row_len(sd0 ? req_s[qs.order[s]] : req_o[qs.order[s]]);
                }
                run_rows = (l != 0 && run_rows > kSat / l) ? kSat : run_rows * l;
                qs.rows[s] = (int64_t)run_rows;
                qs.kind[s] = GSMAT_STEP_PRODUCT;
            }
        } else {
            DevBuf off, fr, ln;
            GS_TRY(off.alloc(sizeof(int64_t) * (size_t)(cur.rows + 1), st));
            if (spec.nrow > 0) {
                GS_TRY(fr.alloc(sizeof(int32_t) * (size_t)spec.nrow * (size_t)cur.rows, st));
                GS_TRY(ln.alloc(sizeof(int32_t) * (size_t)spec.nrow * (size_t)cur.rows, st));
            }
            GS_TRY(launch_product_count_scan(S->view, spec, cur.cols(), cur.rows, off.as<int64_t>(), fr.as<int32_t>(),
                                             ln.as<int32_t>(), cx.d_count(), cx.d_err(), st));
            GS_TRY(cx.read_count(&total));
            if (total > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "product of %lld rows", (long long)total);
            if (!count_rows && total > 0) {
                OutCols oc;
                GS_TRY(alloc_cols(nxt, col, total, st, &oc));
                GS_TRY(launch_product(S->view, spec, cur.cols(), cur.ncols, cur.rows, off.as<int64_t>(),
                                      fr.as<int32_t>(), ln.as<int32_t>(), total, oc, st, S->tiles));
            }
            // intermediates of the fused steps are not built
            for (int s = a; s < b; ++s) {
                qs.rows[s] = s == b - 1 ? total : -1;
                qs.kind[s] = GSMAT_STEP_PRODUCT;
            }
        }
        nxt.rows = total;
        nxt.ncols = col;
        cur = std::move(nxt);
        return GSMAT_OK;
    };
    int first = 0;
    if (fixed_prefix >= 2 && cur.rows > 0) {
        // the constant rows' product, in variable order
        GS_TRY(product_segment(0, fixed_prefix, false));
        first = fixed_prefix;
    }
    for (int step = first; step < tail && cur.rows > 0; ++step) {
        const gsmat_pattern &p = pats[qs.order[step]];
        const int kind = qs.kind[step];
        const PredSide &ps0 = S->side[0][slot[qs.order[step]]];
        const PredSide &ps1 = S->side[1][slot[qs.order[step]]];
        const bool last = step == n_pats - 1;
        const bool unit = cur.rows == 1 && cur.ncols == 0;
        Tbl nxt;
        if (fused[step]) {
            // already applied by the intersect-expand of an earlier step
            qs.kind[step] = GSMAT_STEP_FUSED;
            qs.rows[step] = cur.rows;
            continue;
        }
        if (partner[step] >= 0) {
            const gsmat_pattern &f = pats[qs.order[partner[step]]];
            const int fslot = slot[qs.order[partner[step]]];
            const int side_a = kind == GSMAT_STEP_EXPAND_S ? 0 : 1;
            const PredSide &pa = side_a == 0 ? ps0 : ps1;
            const int32_t known = side_a == 0 ? p.s : p.o;
            const int32_t newv = side_a == 0 ? p.o : p.s;
            ValueSrc a{cur.col[cur.col_of(known)], 0};
            // the filter's other end selects v's candidates: (v f b) -> the
            // row of b by object lists subjects; (b f v) -> by subject
            const bool v_is_s = f.s_var && f.s == newv;
            const int side_b = v_is_s ? 1 : 0;
            const bool b_var = v_is_s ? f.o_var : f.s_var;
            const int32_t b_id = v_is_s ? f.o : f.s;
            ValueSrc b{b_var ? cur.col[cur.col_of(b_id)] : nullptr, b_var ? 0 : b_id};
            const PredSide &pb = S->side[side_b][fslot];
            DevBuf cnt, off;
            GS_TRY(cnt.alloc(sizeof(int32_t) * (size_t)cur.rows, st));
            GS_TRY(off.alloc(sizeof(int64_t) * (size_t)(cur.rows + 1), st));
            GS_TRY(launch_isect_count(S->view, side_a, pa, a, side_b, pb, b, cur.rows, cnt.as<int32_t>(), st));
            GS_TRY(exclusive_scan_i32(cnt.as<int32_t>(), off.as<int64_t>(), cur.rows, st, cx.d_err()));
            GS_CUDA(cudaMemcpyAsync(cx.d_count(), off.as<int64_t>() + cur.rows, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
            int64_t total = 0;
            GS_TRY(cx.read_count(&total));
            if (total > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "step %d: %lld rows", step, (long long)total);
            bool last_live = true;  // every later step runs inside this one
            for (int t = step + 1; t < n_pats; ++t) {
                if (!fused[t]) last_live = false;
            }
            if (count_only && last_live) {
                nxt.rows = total;
                nxt.ncols = cur.ncols + 1;
            } else {
                OutCols oc;
                GS_TRY(alloc_cols(nxt, cur.ncols + 1, total, st, &oc));
                GS_TRY(launch_isect_write(S->view, side_a, pa, a, side_b, pb, b, cur.rows, off.as<int64_t>(), cur.cols(),
                                          cur.ncols, total, oc, st));
            }
            for (int c = 0; c < cur.ncols; ++c) nxt.vars[c] = cur.vars[c];
            nxt.vars[cur.ncols] = newv;
            qs.kind[step] = GSMAT_STEP_INTERSECT;
            cur = std::move(nxt);
            qs.rows[step] = cur.rows;
            continue;
        }
        if (kind == GSMAT_STEP_FILTER) {
            ValueSrc vs{p.s_var ? cur.col[cur.col_of(p.s)] : nullptr, p.s_var ? 0 : p.s};
            ValueSrc vo{p.o_var ? cur.col[cur.col_of(p.o)] : nullptr, p.o_var ? 0 : p.o};
            OutCols oc;
            const int keep = (count_only && last) ? 0 : cur.ncols;
            GS_TRY(alloc_cols(nxt, cur.ncols, cur.rows, st, &oc));
            GS_TRY(launch_filter(S->view, ps0, ps1, vs, vo, cur.cols(), keep, cur.rows, oc, cx.d_count(), cx.d_err(), st,
                                 S->tiles));
            int64_t cnt = 0;
            GS_TRY(cx.read_count(&cnt));
            nxt.rows = cnt;
            for (int c = 0; c < cur.ncols; ++c) nxt.vars[c] = cur.vars[c];
        } else if (kind == GSMAT_STEP_EXPAND_S || kind == GSMAT_STEP_EXPAND_O) {
            const int side = kind == GSMAT_STEP_EXPAND_S ? 0 : 1;
            const PredSide &ps = side == 0 ? ps0 : ps1;
            const bool from_var = side == 0 ? p.s_var : p.o_var;
            const int32_t known = side == 0 ? p.s : p.o;
            const int32_t newv = side == 0 ? p.o : p.s;
            if (!from_var) {
                // a constant's row: Cartesian product with it
                const int r = side == 0 ? req_s[qs.order[step]] : req_o[qs.order[step]];
                const int64_t first = rng[2 * r], m = row_len(r);
                Cols rel;
                rel.c[0] = S->view.side[side].val + first;
                if (unit) {
                    nxt.rows = m;
                    nxt.ncols = 1;
                    nxt.col[0] = rel.c[0];
                } else {
                    const int64_t total = cur.rows * m;
                    if (total > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "step %d: %lld rows", step, (long long)total);
                    if (count_only && last) {
                        nxt.rows = total;
                        nxt.ncols = cur.ncols + 1;
                    } else {
                        OutCols oc;
                        GS_TRY(alloc_cols(nxt, cur.ncols + 1, total, st, &oc));
                        GS_TRY(launch_cross(cur.cols(), cur.ncols, cur.rows, rel, 1, m, oc, st));
                    }
                }
                for (int c = 0; c < cur.ncols; ++c) nxt.vars[c] = cur.vars[c];
                nxt.vars[cur.ncols] = newv;
            } else {
                const int xc = cur.col_of(known);
                DevBuf off, fst;
                GS_TRY(off.alloc(sizeof(int64_t) * (size_t)(cur.rows + 1), st));
                GS_TRY(fst.alloc(sizeof(int32_t) * (size_t)cur.rows, st));
                GS_TRY(launch_count_scan(S->view, side, ps, cur.col[xc], cur.rows, off.as<int64_t>(), fst.as<int32_t>(),
                                         cx.d_count(), cx.d_err(), st));
                int64_t total = 0;
                GS_TRY(cx.read_count(&total));
                if (total > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "step %d: %lld rows", step, (long long)total);
                if (count_only && last) {
                    nxt.rows = total;
                    nxt.ncols = cur.ncols + 1;
                } else {
                    OutCols oc;
                    GS_TRY(alloc_cols(nxt, cur.ncols + 1, total, st, &oc));
                    GS_TRY(launch_expand(S->view, side, cur.cols(), cur.ncols, cur.rows, off.as<int64_t>(),
                                         fst.as<int32_t>(), total, oc, st, S->tiles));
                }
                for (int c = 0; c < cur.ncols; ++c) nxt.vars[c] = cur.vars[c];
                nxt.vars[cur.ncols] = newv;
            }
        } else {  // CROSS
            Cols rel;
            int rc;
            int64_t m = 0;
            DevBuf diag;
            int32_t rv[2];
            if (p.s == p.o) {  // ?x p ?x
                GS_TRY(diag.alloc(sizeof(int32_t) * (size_t)(ps0.nnz > 0 ? ps0.nnz : 1), st));
                GS_TRY(launch_diag(S->view, ps0, diag.as<int32_t>(), cx.d_count(), cx.d_err(), st));
                GS_TRY(cx.read_count(&m));
                rel.c[0] = diag.as<int32_t>();
                rc = 1;
                rv[0] = p.s;
            } else {
                // M_p from whichever side puts the lower variable id first:
                // rows by subject are (s, o)-ascending, rows by object
                // (o, s)-ascending, so the result stays sorted and the final
                // reorder to variable order has less to do
                const int sd = p.o < p.s ? 1 : 0;
                const PredSide &pss = sd == 0 ? ps0 : ps1;
                rel.c[0] = S->view.side[sd].key + pss.ent_base;
                rel.c[1] = S->view.side[sd].val + pss.ent_base;
                m = pss.nnz;
                rc = 2;
                rv[0] = sd == 0 ? p.s : p.o;
                rv[1] = sd == 0 ? p.o : p.s;
            }
            if (unit) {
                nxt.rows = m;
                nxt.ncols = rc;
                for (int c = 0; c < rc; ++c) nxt.col[c] = rel.c[c];
                nxt.buf = std::move(diag);  // owns the diagonal when there is one
            } else {
                const int64_t total = cur.rows * m;
                if (total > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "step %d: %lld rows", step, (long long)total);
                if (count_only && last) {
                    nxt.rows = total;
                    nxt.ncols = cur.ncols + rc;
                } else {
                    OutCols oc;
                    GS_TRY(alloc_cols(nxt, cur.ncols + rc, total, st, &oc));
                    GS_TRY(launch_cross(cur.cols(), cur.ncols, cur.rows, rel, rc, m, oc, st));
                }
            }
            for (int c = 0; c < cur.ncols; ++c) nxt.vars[c] = cur.vars[c];
            for (int c = 0; c < rc; ++c) nxt.vars[cur.ncols + c] = rv[c];
        }
        cur = std::move(nxt);
        if (step == 0 && n_shards > 1) {
            // row sharding: keep this shard's contiguous part of the first
            // relation; every later step maps each row to rows of its own, in
            // order, so the shards partition the result
            const int64_t lo = cur.rows * shard / n_shards, hi = cur.rows * (shard + 1) / n_shards;
            for (int c = 0; c < cur.ncols; ++c) cur.col[c] += lo;
            cur.rows = hi - lo;
        }
        qs.rows[step] = cur.rows;
    }

    if (tail < n_pats && cur.rows > 0) GS_TRY(product_segment(tail, n_pats, count_only));

    // result
    const int64_t rows = cur.rows;
    qs.result_rows = rows;
    if (count_only) {
        T->rows = rows;
        T->ncols = 0;
        return GSMAT_OK;
    }
    if (rows == 0 || cur.ncols != n_vars) {
        // empty result (possibly before every variable was bound)
        T->rows = 0;
        T->ncols = n_vars;
        for (int c = 0; c < n_vars; ++c) {
            T->vars[c] = (flags & GSMAT_PLAN_ORDER) ? plan_vars[c] : c;
            T->col[c] = nullptr;
        }
        return GSMAT_OK;
    }
    Tbl fin;
    if (flags & GSMAT_PLAN_ORDER) {
        fin.rows = cur.rows;
        fin.ncols = cur.ncols;
        for (int c = 0; c < cur.ncols; ++c) {
            fin.vars[c] = cur.vars[c];
            fin.col[c] = cur.col[c];
        }
        fin.buf = std::move(cur.buf);
    } else {
        GS_TRY(canonical_order(cx, cur, fin));
    }
    // the result owns its columns (a view of the store is copied)
    if (!fin.buf.p && fin.ncols > 0) {
        Tbl own;
        OutCols oc;
        GS_TRY(alloc_cols(own, fin.ncols, fin.rows, st, &oc));
        GS_TRY(launch_copy_cols(fin.cols(), fin.ncols, fin.rows, oc, st));
        for (int c = 0; c < fin.ncols; ++c) own.vars[c] = fin.vars[c];
        fin = std::move(own);
    }
    T->rows = fin.rows;
    T->ncols = fin.ncols;
    for (int c = 0; c < fin.ncols; ++c) {
        T->vars[c] = fin.vars[c];
        T->col[c] = fin.col[c];
    }
    T->storage = std::move(fin.buf);
    // wait for the reorder or copy, whose bounded waits report into the same
    // error word (the earlier returns follow a read of the last step's count)
    int64_t unused = 0;
    GS_TRY(cx.read_count(&unused));
    return GSMAT_OK;
}

}  // namespace

int query_run(const gsmat_store *S, const gsmat_pattern *pats, int n_pats, int n_vars, uint32_t flags, cudaStream_t st,
              gsmat_table **out, int shard, int n_shards) {
    if (!S || !out) return set_error(GSMAT_ERR_INVALID_ARG, "store or out is NULL");
    *out = nullptr;
    if (n_shards < 1 || n_shards > (1 << 20) || shard < 0 || shard >= n_shards) {
        return set_error(GSMAT_ERR_INVALID_ARG, "shard %d of %d", shard, n_shards);
    }
    gsmat_table *T = new gsmat_table();
    // on success run() has waited for its last device work (its final read
    // of the error word); a failed call drains what it enqueued
    const int rc = run(S, pats, n_pats, n_vars, flags, st, T, shard, n_shards);
    if (rc != GSMAT_OK) cudaStreamSynchronize(st);
    profile_flush();
    if (rc != GSMAT_OK) {
        delete T;
        return rc;
    }
    T->storage.st = nullptr;  // freed on the legacy stream later
    *out = T;
    return GSMAT_OK;
}

int store_tune(gsmat_store *S, const gsmat_bgp *bgps, int32_t n, cudaStream_t st, TileConfig *best) {
    if (!S || !bgps || n < 1 || !best) return set_error(GSMAT_ERR_INVALID_ARG, "store tune: bad arguments");
    for (int32_t i = 0; i < n; ++i) GS_TRY(validate_bgp(bgps[i].pats, bgps[i].n_pats, bgps[i].n_vars));
    const TileConfig keep = S->tiles;
    std::vector<TileConfig> cands;
    cands.push_back(TileConfig());  // the default first: a tie keeps it
    for (int e : {512, 1024, 2048, 4096, 8192}) {
        for (int r : {16, 64, 256}) {
            TileConfig c;
            c.expand_items = e;
            c.short_row = r;
            if (c.expand_items != cands[0].expand_items || c.short_row != cands[0].short_row) cands.push_back(c);
        }
    }
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return set_error(GSMAT_ERR_CUDA, "store tune: events");
    }
    auto run_all = [&]() -> int {
        for (int32_t i = 0; i < n; ++i) {
            gsmat_table *T = nullptr;
            GS_TRY(query_run(S, bgps[i].pats, bgps[i].n_pats, bgps[i].n_vars, GSMAT_SORTED, st, &T, 0, 1));
            delete T;
        }
        return GSMAT_OK;
    };
    int rc = GSMAT_OK;
    double best_ms = 1e300;
    TileConfig pick = cands[0];
    for (const TileConfig &c : cands) {
        S->tiles = c;
        if ((rc = run_all()) != GSMAT_OK) break;  // warm-up (allocator pool, caches)
        double ms_min = 1e300;
        for (int rep = 0; rep < 2 && rc == GSMAT_OK; ++rep) {
            cudaEventRecord(a, st);
            rc = run_all();
            cudaEventRecord(b, st);
            float ms = 0;
            if (rc == GSMAT_OK && (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess)) {
                rc = set_error(GSMAT_ERR_CUDA, "store tune: timing");
            }
            ms_min = std::min(ms_min, (double)ms);
        }
        if (rc != GSMAT_OK) break;
        if (ms_min < best_ms) {
            best_ms = ms_min;
            pick = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != GSMAT_OK) {
        S->tiles = keep;
        return rc;
    }
    S->tiles = pick;
    *best = pick;
    return GSMAT_OK;
}

int reorder_view(const gsmat_store *S, const int32_t *const *plan_cols, const int32_t *plan_vars, int V, int64_t rows,
                 cudaStream_t st, gsmat_table **out) {
    *out = nullptr;
    Ctx cx;
    cx.S = S;
    cx.st = st;
    cx.h = pinned_scratch(4 + 8 * GSMAT_MAX_PATTERNS);
    if (!cx.h) return set_error(GSMAT_ERR_CUDA, "pinned host scratch");
    GS_TRY(cx.qstat.alloc(4 * sizeof(int64_t), st));
    GS_CUDA(cudaMemsetAsync(cx.qstat.p, 0, 4 * sizeof(int64_t), st));
    Tbl t;
    t.rows = rows;
    t.ncols = V;
    for (int c = 0; c < V; ++c) {
        t.col[c] = plan_cols[c];
        t.vars[c] = plan_vars[c];
    }
    Tbl fin;
    GS_TRY(canonical_order(cx, t, fin));
    gsmat_table *T = new gsmat_table();
    T->rows = fin.rows;
    T->ncols = fin.ncols;
    for (int c = 0; c < fin.ncols; ++c) {
        T->vars[c] = fin.vars[c];
        T->col[c] = fin.col[c];
    }
    T->storage = std::move(fin.buf);
    T->stats.result_rows = fin.rows;
    T->id_bits = std::max(1, bits_for((uint64_t)std::max(S->max_entity, 0)));
    int64_t unused = 0;
    const int rc = cx.read_count(&unused);  // waits for the reorder, checks its bounded waits
    if (rc != GSMAT_OK) {
        cudaStreamSynchronize(st);
        delete T;
        return rc;
    }
    T->storage.st = nullptr;
    *out = T;
    return GSMAT_OK;
}

namespace {

// Row i is the first of its run of equal rows (rows sorted, k columns).
struct FirstOfRunOp {
    Cols in;
    OutCols out;
    int k;
    __device__ bool flag(int64_t i) const {
        if (i == 0) return true;
        for (int c = 0; c < k; ++c) {
            if (in.c[c][i] != in.c[c][i - 1]) return true;
        }
        return false;
    }
    __device__ void emit(int64_t i, int64_t j) const {
        for (int c = 0; c < k; ++c) out.c[c][j] = in.c[c][i];
    }
};

// -1, 0, 1: row ia of A against row ib of B, lexicographically over V columns
__device__ __forceinline__ int cmp_rows(const Cols &A, int64_t ia, const Cols &B, int64_t ib, int V) {
    for (int c = 0; c < V; ++c) {
        const int32_t x = A.c[c][ia], y = B.c[c][ib];
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}

// *flag = 1 if some row of the n-row table is below its predecessor.
__global__ void __launch_bounds__(256) unsorted_kernel(Cols A, int64_t n, int V, int *flag) {
    for (int64_t i = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (cmp_rows(A, i - 1, A, i, V) > 0) {
            *flag = 1;
            return;
        }
    }
}

// Merge path: thread t writes outputs [16 t, 16 t + 16) of the merge of the
// sorted tables A (nA rows) and B (nB rows), A's row first among equal ones.
// A binary search on the cross diagonal gives how many of the first 16 t
// outputs come from A; the thread then merges sequentially from there.
constexpr int kMergeItems = 16;
__global__ void __launch_bounds__(256) merge2_kernel(Cols A, int64_t nA, Cols B, int64_t nB, int V, OutCols C) {
    const int64_t total = nA + nB;
    const int64_t d0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kMergeItems;
    if (d0 >= total) return;
    int64_t lo = d0 > nB ? d0 - nB : 0, hi = d0 < nA ? d0 : nA;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;  // mid < nA, 0 <= d0 - 1 - mid < nB
        if (cmp_rows(A, mid, B, d0 - 1 - mid, V) <= 0) lo = mid + 1;
        else hi = mid;
    }
    int64_t i = lo, j = d0 - lo;
    const int64_t d1 = d0 + kMergeItems < total ? d0 + kMergeItems : total;
    for (int64_t d = d0; d < d1; ++d) {
        if (i < nA && (j >= nB || cmp_rows(A, i, B, j, V) <= 0)) {
            for (int c = 0; c < V; ++c) C.c[c][d] = A.c[c][i];
            ++i;
        } else {
            for (int c = 0; c < V; ++c) C.c[c][d] = B.c[c][j];
            ++j;
        }
    }
}

}  // namespace

int table_project(const gsmat_table *T, const int32_t *vars, int32_t n, int distinct, cudaStream_t st,
                  gsmat_table **out) {
    if (!T || !vars || !out) return set_error(GSMAT_ERR_INVALID_ARG, "table, vars or out is NULL");
    *out = nullptr;
    if (T->ncols == 0) return set_error(GSMAT_ERR_INVALID_ARG, "a count-only table has no columns");
    if (n < 1 || n > T->ncols) return set_error(GSMAT_ERR_INVALID_ARG, "%d projected variables (1..%d)", n, T->ncols);
    if (distinct != 0 && distinct != 1) return set_error(GSMAT_ERR_INVALID_ARG, "distinct must be 0 or 1");
    int idx[kMaxCols];
    bool leading = true;  // the new columns are the table's first n, in order
    for (int c = 0; c < n; ++c) {
        idx[c] = -1;
        for (int j = 0; j < T->ncols; ++j) {
            if (T->vars[j] == vars[c]) idx[c] = j;
        }
        if (idx[c] < 0) return set_error(GSMAT_ERR_INVALID_ARG, "variable %d is not a column of the table", vars[c]);
        for (int b = 0; b < c; ++b) {
            if (idx[b] == idx[c]) return set_error(GSMAT_ERR_INVALID_ARG, "variable %d projected twice", vars[c]);
        }
        leading = leading && idx[c] == c;
    }
    const int64_t rows = T->rows;
    auto fill = [&](gsmat_table *R, int64_t r) {
        R->rows = r;
        R->ncols = n;
        R->id_bits = T->id_bits;
        R->stats.result_rows = r;
        for (int c = 0; c < n; ++c) R->vars[c] = vars[c];
    };
    if (rows == 0) {
        gsmat_table *R = new gsmat_table();
        fill(R, 0);
        *out = R;
        return GSMAT_OK;
    }
    Ctx cx;
    cx.S = nullptr;
    cx.st = st;
    cx.h = pinned_scratch(4 + 8 * GSMAT_MAX_PATTERNS);
    if (!cx.h) return set_error(GSMAT_ERR_CUDA, "pinned host scratch");
    GS_TRY(cx.qstat.alloc(4 * sizeof(int64_t), st));
    GS_CUDA(cudaMemsetAsync(cx.qstat.p, 0, 4 * sizeof(int64_t), st));
    Cols in;
    for (int c = 0; c < kMaxCols; ++c) in.c[c] = c < n ? T->col[idx[c]] : nullptr;
    // rows of the table ascend in its column order, so its leading columns
    // are already sorted; other selections are reordered (stable LSD)
    Tbl srt;
    if (!leading || !distinct) {
        OutCols oc;
        GS_TRY(alloc_cols(srt, n, rows, st, &oc));
        if (leading) {
            GS_TRY(launch_copy_cols(in, n, rows, oc, st));
        } else {
            GS_TRY(reorder_rows(in, n, n, std::max(1, T->id_bits), rows, oc, st, cx.d_err()));
        }
        in = srt.cols();
    }
    int64_t kept = rows;
    Tbl res;
    if (distinct) {
        OutCols oc;
        GS_TRY(alloc_cols(res, n, rows, st, &oc));
        FirstOfRunOp op{in, oc, n};
        GS_TRY(run_select(op, rows, cx.d_count(), st, cx.d_err()));
        GS_TRY(cx.read_count(&kept));  // waits for the device, checks its bounded waits
    } else {
        res = std::move(srt);
        int64_t unused = 0;
        GS_TRY(cx.read_count(&unused));
    }
    gsmat_table *R = new gsmat_table();
    fill(R, kept);
    for (int c = 0; c < n; ++c) R->col[c] = res.col[c];
    R->storage = std::move(res.buf);
    R->storage.st = nullptr;  // freed on the legacy stream later
    *out = R;
    return GSMAT_OK;
}

int table_merge(const gsmat_table *const *tables, int k, cudaStream_t st, gsmat_table **out) {
    if (!tables || !out || k < 1) return set_error(GSMAT_ERR_INVALID_ARG, "tables, k or out");
    *out = nullptr;
    const gsmat_table *t0 = tables[0];
    if (!t0 || t0->ncols == 0) return set_error(GSMAT_ERR_INVALID_ARG, "table 0 is NULL or has no columns");
    const int V = t0->ncols;
    int64_t total = 0;
    int bits = 1;
    for (int i = 0; i < k; ++i) {
        const gsmat_table *t = tables[i];
        if (!t || t->ncols != V) return set_error(GSMAT_ERR_INVALID_ARG, "table %d: other columns", i);
        for (int c = 0; c < V; ++c) {
            if (t->vars[c] != t0->vars[c]) return set_error(GSMAT_ERR_INVALID_ARG, "table %d: other variables", i);
        }
        total += t->rows;
        bits = std::max(bits, t->id_bits);
    }
    if (total > (int64_t)UINT32_MAX) return set_error(GSMAT_ERR_CAPACITY, "%lld rows", (long long)total);
    gsmat_table *R = new gsmat_table();
    R->ncols = V;
    R->id_bits = bits;
    for (int c = 0; c < V; ++c) R->vars[c] = t0->vars[c];
    if (total == 0) {
        *out = R;
        return GSMAT_OK;
    }
    auto fail = [&](int rc) {
        cudaStreamSynchronize(st);
        delete R;
        return rc;
    };
    Ctx cx;
    cx.S = nullptr;
    cx.st = st;
    cx.h = pinned_scratch(4 + 8 * GSMAT_MAX_PATTERNS);
    if (!cx.h) return fail(set_error(GSMAT_ERR_CUDA, "pinned host scratch"));
    int rc = cx.qstat.alloc(4 * sizeof(int64_t), st);
    if (rc != GSMAT_OK) return fail(rc);
    if (cudaMemsetAsync(cx.qstat.p, 0, 4 * sizeof(int64_t), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(set_error(GSMAT_ERR_CUDA, "memset"));
    }
    struct Run {
        Cols cols;
        int64_t rows = 0;
        Tbl own;  // the columns' storage; empty for an input table
    };
    std::vector<Run> runs;
    for (int i = 0; i < k; ++i) {
        if (tables[i]->rows == 0) continue;
        Run r;
        for (int c = 0; c < kMaxCols; ++c) r.cols.c[c] = c < V ? tables[i]->col[c] : nullptr;
        r.rows = tables[i]->rows;
        runs.push_back(std::move(r));
    }
    // are the tables sorted (as query results are)?  then merge them
    // pairwise by merge path; otherwise put them back to back and reorder
    int *d_flag = reinterpret_cast<int *>(cx.qstat.as<int64_t>() + 2);
    for (const Run &r : runs) {
        if (r.rows < 2) continue;
        unsorted_kernel<<<grid_1d(r.rows, 256), 256, 0, st>>>(r.cols, r.rows, V, d_flag);
        GS_LAUNCH_CHECK();
    }
    if ((rc = read_words(cx.qstat.p, cx.h, 3, st)) != GSMAT_OK) return fail(rc);
    const bool sorted = reinterpret_cast<const int *>(cx.h + 2)[0] == 0;
    Tbl res;
    OutCols ro;
    if (!sorted) {
        Tbl cat;
        OutCols oc;
        if ((rc = alloc_cols(cat, V, total, st, &oc)) != GSMAT_OK) return fail(rc);
        int64_t at = 0;
        for (const Run &r : runs) {
            OutCols dst;
            for (int c = 0; c < kMaxCols; ++c) dst.c[c] = c < V ? oc.c[c] + at : nullptr;
            if ((rc = launch_copy_cols(r.cols, V, r.rows, dst, st)) != GSMAT_OK) return fail(rc);
            at += r.rows;
        }
        if ((rc = alloc_cols(res, V, total, st, &ro)) != GSMAT_OK) return fail(rc);
        if ((rc = reorder_rows(cat.cols(), V, V, bits, total, ro, st, cx.d_err())) != GSMAT_OK) return fail(rc);
    } else if (runs.size() == 1) {
        if ((rc = alloc_cols(res, V, total, st, &ro)) != GSMAT_OK) return fail(rc);
        if ((rc = launch_copy_cols(runs[0].cols, V, total, ro, st)) != GSMAT_OK) return fail(rc);
    } else {
        // rounds of pairwise merges (the odd run waits a round, keeping its
        // storage); replacing a round's runs frees the merged inputs, in
        // stream order after the merges that read them
        while (runs.size() > 1) {
            std::vector<Run> next;
            for (size_t a = 0; a + 1 < runs.size(); a += 2) {
                const Run &A = runs[a], &B = runs[a + 1];
                Run m;
                m.rows = A.rows + B.rows;
                OutCols oc;
                if ((rc = alloc_cols(m.own, V, m.rows, st, &oc)) != GSMAT_OK) return fail(rc);
                // one thread per kMergeItems outputs, no grid cap
                const int64_t threads = (m.rows + kMergeItems - 1) / kMergeItems;
                const unsigned blocks = (unsigned)((threads + 255) / 256);
                merge2_kernel<<<blocks, 256, 0, st>>>(A.cols, A.rows, B.cols, B.rows, V, oc);
                GS_LAUNCH_CHECK();
                m.cols = m.own.cols();
                next.push_back(std::move(m));
            }
            if (runs.size() % 2) next.push_back(std::move(runs.back()));
            runs = std::move(next);
        }
        res = std::move(runs[0].own);  // made by the last merge
    }
    int64_t unused = 0;
    if ((rc = cx.read_count(&unused)) != GSMAT_OK) return fail(rc);
    R->rows = total;
    R->stats.result_rows = total;
    for (int c = 0; c < V; ++c) R->col[c] = res.col[c];
    R->storage = std::move(res.buf);
    R->storage.st = nullptr;  // freed on the legacy stream later
    *out = R;
    return GSMAT_OK;
}

int table_copy(const gsmat_table *T, int32_t *dst, int dst_on_device, cudaStream_t st, bool sync) {
    if (!T || (!dst && T->rows > 0 && T->ncols > 0)) return set_error(GSMAT_ERR_INVALID_ARG, "table or dst is NULL");
    const int64_t n = T->rows;
    const int k = T->ncols;
    if (n == 0 || k == 0) return GSMAT_OK;
    Cols in;
    for (int c = 0; c < kMaxCols; ++c) in.c[c] = c < k ? T->col[c] : nullptr;
    if (dst_on_device) {
        GS_TRY(launch_interleave(in, k, n, dst, st));
        if (sync) GS_CUDA(cudaStreamSynchronize(st));
        return GSMAT_OK;
    }
    DevBuf tmp;  // freed in stream order after the copy
    GS_TRY(tmp.alloc(sizeof(int32_t) * (size_t)n * k, st));
    GS_TRY(launch_interleave(in, k, n, tmp.as<int32_t>(), st));
    GS_CUDA(cudaMemcpyAsync(dst, tmp.p, sizeof(int32_t) * (size_t)n * k, cudaMemcpyDeviceToHost, st));
    if (sync) GS_CUDA(cudaStreamSynchronize(st));
    return GSMAT_OK;
}

}  // namespace gs
