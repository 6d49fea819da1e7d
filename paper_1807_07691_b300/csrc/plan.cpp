// Host query planner: Alg. 1 ("Query Plan Generated", Sec. 6.2.2) and the
// accumulated intermediate-size estimate of Sec. 6.2.1.
//
// Alg. 1 as printed resets its scan index on every iteration and removes a
// pattern in both branches; the prose of Sec. 6.2.1 (steps 1-4) is followed:
//  1. sort the patterns by their statistic (stable: ties keep input order);
//  2. take the smallest;
//  3. take, in sorted order, the first remaining pattern that shares a
//     variable with the patterns taken so far (constants do not connect);
//  4. repeat; if no remaining pattern shares a variable (a disconnected
//     BGP), take the smallest remaining one -- a Cartesian product.
// The estimate starts from 1 and multiplies, per step, by the key (CROSS,
// or EXPAND from a constant), by the average row size nnz / nr on the bound
// side (EXPAND from a variable), or by min(1, nnz / (nr_s * nr_o)) (FILTER);
// the cost is the sum of the running estimates, the quantity Thm. 1 and
// Thm. 2 bound.
//
// Alg. 1 is greedy: it fixes the first pattern by its statistic alone and
// never revisits a choice.  The cost-based variant keeps the estimate and
// the connectivity rule but minimises the cost itself: over every connected
// order of a BGP of at most kCostPlanMax patterns (each step takes a
// pattern sharing a variable with those taken, unless none remains that
// does), it returns one of least cost; among equal costs, the one whose
// sequence of positions in the key order is smallest, which makes Alg. 1's
// order the winner of any tie it is part of.
#include <string.h>

#include <algorithm>
#include <limits>
#include <vector>

#include "plan.h"

namespace gs {

namespace {

uint64_t vars_of(const gsmat_pattern &p) {
    uint64_t m = 0;
    if (p.s_var) m |= uint64_t(1) << p.s;
    if (p.o_var) m |= uint64_t(1) << p.o;
    return m;
}

// Running-estimate factor of a pattern taken as a step of the given kind.
double step_factor(const gsmat_pattern &p, int kind, int64_t key, const gsmat_pred_stats &st) {
    const double nnz = (double)st.nnz, nr_s = (double)st.nr_s, nr_o = (double)st.nr_o;
    if (kind == GSMAT_STEP_CROSS) return (double)key;
    if (kind == GSMAT_STEP_FILTER) return (nr_s > 0 && nr_o > 0) ? std::min(1.0, nnz / (nr_s * nr_o)) : 0.0;
    if (kind == GSMAT_STEP_EXPAND_S) return !p.s_var ? (double)key : (nr_s > 0 ? nnz / nr_s : 0.0);
    return !p.o_var ? (double)key : (nr_o > 0 ? nnz / nr_o : 0.0);
}

}  // namespace

int step_kind(const gsmat_pattern &p, uint64_t bound) {
    const bool s_known = !p.s_var || ((bound >> p.s) & 1);
    const bool o_known = !p.o_var || ((bound >> p.o) & 1);
    if (s_known && o_known) return GSMAT_STEP_FILTER;
    if (s_known) return GSMAT_STEP_EXPAND_S;
    if (o_known) return GSMAT_STEP_EXPAND_O;
    return GSMAT_STEP_CROSS;
}

int plan_bgp(const gsmat_pattern *pats, int n, const int64_t *keys, const gsmat_pred_stats *stats, int32_t *order,
             int32_t *kinds, double *est) {
    std::vector<int> L(n);
    for (int i = 0; i < n; ++i) L[i] = i;
    std::stable_sort(L.begin(), L.end(), [&](int a, int b) { return keys[a] < keys[b]; });
    uint64_t N = 0;
    for (int step = 0; step < n; ++step) {
        size_t pick = 0;
        if (step > 0) {
            pick = L.size();
            for (size_t t = 0; t < L.size(); ++t) {
                if (vars_of(pats[L[t]]) & N) {
                    pick = t;
                    break;
                }
            }
            if (pick == L.size()) pick = 0;
        }
        order[step] = L[pick];
        N |= vars_of(pats[L[pick]]);
        L.erase(L.begin() + (long)pick);
    }
    uint64_t bound = 0;
    double e = 1.0;
    for (int step = 0; step < n; ++step) {
        const int i = order[step];
        const gsmat_pattern &p = pats[i];
        const int kind = step_kind(p, bound);
        e = e * step_factor(p, kind, keys[i], stats[i]);
        if (kinds) kinds[step] = kind;
        if (est) est[step] = e;
        bound |= vars_of(p);
    }
    return GSMAT_OK;
}

namespace {

// Depth-first search over the connected orders (an order is connected when
// each step takes a pattern sharing a variable with those already taken,
// unless no remaining pattern does), branching on the remaining patterns in
// the key order of Alg. 1, so the first complete order reached is Alg. 1's.
// An order replaces the best one only when its cost is strictly smaller;
// since every running estimate is >= 0, a prefix whose partial sum already
// reaches the best cost cannot lead to a strictly smaller one and is cut.
struct CostSearch {
    const gsmat_pattern *pats;
    const int64_t *keys;
    const gsmat_pred_stats *stats;
    int n;
    int L[kCostPlanMax];        // pattern indices in key order
    uint64_t vm[kCostPlanMax];  // variables of L[t]
    int cur[kCostPlanMax];
    int best_order[kCostPlanMax];
    double fmin[kCostPlanMax];  // least factor L[t] can contribute as any step
    double best;

    // Lower bound on what the remaining patterns add to the cost from a
    // running estimate e: every factor is at least its pattern's fmin, and
    // a product of positive factors is at least the product of as many of
    // the smallest fmin, so the k-th remaining running estimate is at least
    // e times the k smallest fmin.  Scaled down by 1e-9 so that rounding
    // never cuts an order that is cheaper by less than that.
    double remaining_bound(unsigned taken, double e) const {
        double f[kCostPlanMax];
        int r = 0;
        for (int t = 0; t < n; ++t) {
            if ((taken >> t) & 1) continue;
            int j = r++;
            for (; j > 0 && f[j - 1] > fmin[t]; --j) f[j] = f[j - 1];
            f[j] = fmin[t];
        }
        double sum = 0.0, run = e;
        for (int k = 0; k < r; ++k) {
            run *= f[k];
            sum += run;
        }
        return sum * (1.0 - 1e-9);
    }

    void run(int depth, unsigned taken, uint64_t bound, double e, double partial) {
        if (depth == n) {
            if (partial < best) {
                best = partial;
                for (int d = 0; d < n; ++d) best_order[d] = cur[d];
            }
            return;
        }
        if (depth > 0 && depth < n - 1 && !(partial + remaining_bound(taken, e) < best)) return;
        bool connected = false;
        if (depth > 0) {
            for (int t = 0; t < n && !connected; ++t) connected = !((taken >> t) & 1) && (vm[t] & bound);
        }
        for (int t = 0; t < n; ++t) {
            if ((taken >> t) & 1) continue;
            if (connected && !(vm[t] & bound)) continue;
            const int i = L[t];
            const double e2 = e * step_factor(pats[i], step_kind(pats[i], bound), keys[i], stats[i]);
            const double p2 = partial + e2;
            if (!(p2 < best)) continue;
            cur[depth] = i;
            run(depth + 1, taken | (1u << t), bound | vm[t], e2, p2);
        }
    }
};

}  // namespace

int plan_bgp_cost(const gsmat_pattern *pats, int n, const int64_t *keys, const gsmat_pred_stats *stats,
                  int32_t *order, int32_t *kinds, double *est) {
    std::vector<double> greedy_est(n);
    const int rc = plan_bgp(pats, n, keys, stats, order, kinds, greedy_est.data());
    if (rc != GSMAT_OK) return rc;
    if (n > kCostPlanMax) {
        if (est) memcpy(est, greedy_est.data(), sizeof(double) * (size_t)n);
        return GSMAT_OK;
    }
    CostSearch cs;
    cs.pats = pats;
    cs.keys = keys;
    cs.stats = stats;
    cs.n = n;
    for (int i = 0; i < n; ++i) cs.L[i] = i;
    std::stable_sort(cs.L, cs.L + n, [&](int a, int b) { return keys[a] < keys[b]; });
    for (int t = 0; t < n; ++t) cs.vm[t] = vars_of(pats[cs.L[t]]);
    // fmin: the least factor over the step kinds a pattern can take; a
    // variable end can be known beforehand only if another pattern (or the
    // other end of this one) holds the variable too
    int occ[64] = {0};
    for (int i = 0; i < n; ++i) {
        const uint64_t v = vars_of(pats[i]);
        for (int b = 0; b < 64; ++b) occ[b] += (int)((v >> b) & 1);
    }
    for (int t = 0; t < n; ++t) {
        const int i = cs.L[t];
        const gsmat_pattern &p = pats[i];
        const bool s_pre = !p.s_var || occ[p.s] > 1;  // s can be known before this step
        const bool o_pre = !p.o_var || occ[p.o] > 1;
        double f = std::numeric_limits<double>::infinity();
        if (p.s_var && p.o_var) f = std::min(f, step_factor(p, GSMAT_STEP_CROSS, keys[i], stats[i]));
        if (s_pre && p.o_var) f = std::min(f, step_factor(p, GSMAT_STEP_EXPAND_S, keys[i], stats[i]));
        if (o_pre && p.s_var) f = std::min(f, step_factor(p, GSMAT_STEP_EXPAND_O, keys[i], stats[i]));
        if ((s_pre && o_pre) || (p.s_var && p.o_var && p.s == p.o)) {
            f = std::min(f, step_factor(p, GSMAT_STEP_FILTER, keys[i], stats[i]));
        }
        if (!(f >= 0.0) || f == std::numeric_limits<double>::infinity()) f = 0.0;  // no usable bound
        cs.fmin[t] = f;
    }
    // Alg. 1's order is the first connected order of the search: start from
    // it, so that it wins every tie and bounds the search from the outset
    double greedy_cost = 0.0;
    for (int d = 0; d < n; ++d) {
        greedy_cost += greedy_est[d];
        cs.best_order[d] = order[d];
    }
    cs.best = greedy_cost;
    cs.run(0, 0u, 0, 1.0, 0.0);
    // kinds and running estimates of the chosen order
    uint64_t bound = 0;
    double e = 1.0;
    for (int d = 0; d < n; ++d) {
        const int i = cs.best_order[d];
        const int kind = step_kind(pats[i], bound);
        e = e * step_factor(pats[i], kind, keys[i], stats[i]);
        order[d] = i;
        if (kinds) kinds[d] = kind;
        if (est) est[d] = e;
        bound |= vars_of(pats[i]);
    }
    return GSMAT_OK;
}

int validate_bgp(const gsmat_pattern *pats, int n_pats, int n_vars) {
    if (!pats || n_pats < 1 || n_pats > GSMAT_MAX_PATTERNS) {
        return set_error(GSMAT_ERR_INVALID_ARG, "n_pats = %d (1..%d)", n_pats, GSMAT_MAX_PATTERNS);
    }
    if (n_vars < 0 || n_vars > 32) return set_error(GSMAT_ERR_INVALID_ARG, "n_vars = %d (0..32)", n_vars);
    uint64_t used = 0;
    for (int i = 0; i < n_pats; ++i) {
        const gsmat_pattern &p = pats[i];
        if (p.p_var) return set_error(GSMAT_ERR_UNSUPPORTED, "pattern %d has a variable predicate", i);
        if (p.p < 0) return set_error(GSMAT_ERR_INVALID_ARG, "pattern %d: negative predicate id", i);
        const int32_t ends[2] = {p.s, p.o};
        const uint8_t isv[2] = {p.s_var, p.o_var};
        for (int e = 0; e < 2; ++e) {
            if (isv[e]) {
                if (ends[e] < 0 || ends[e] >= n_vars) {
                    return set_error(GSMAT_ERR_INVALID_ARG, "pattern %d: variable %d out of range", i, ends[e]);
                }
                used |= uint64_t(1) << ends[e];
            } else if (ends[e] < 0) {
                return set_error(GSMAT_ERR_INVALID_ARG, "pattern %d: negative constant", i);
            }
        }
    }
    const uint64_t all = n_vars == 0 ? 0 : (n_vars == 64 ? ~uint64_t(0) : ((uint64_t(1) << n_vars) - 1));
    if (used != all) return set_error(GSMAT_ERR_INVALID_ARG, "a variable in 0..%d is used by no pattern", n_vars - 1);
    return GSMAT_OK;
}

}  // namespace gs
