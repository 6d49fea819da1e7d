// Host planner interface (Alg. 1 and the Sec. 6.2 estimate).
#pragma once

#include <stdint.h>

#include "../../include/gsmat.h"

namespace gs {

int set_error(int status, const char *fmt, ...);

// GSMAT_STEP_* of pattern p given the set of bound variables (bit mask).
int step_kind(const gsmat_pattern &p, uint64_t bound);

// Alg. 1 order, step kinds and running estimates (see plan.cpp).
int plan_bgp(const gsmat_pattern *pats, int n, const int64_t *keys, const gsmat_pred_stats *stats, int32_t *order,
             int32_t *kinds, double *est);

// Largest BGP the cost-based variant searches exhaustively.
constexpr int kCostPlanMax = GSMAT_PLAN_COST_MAX;

// Cost-based variant: the connected order of least estimated cost (sum of
// the running estimates), Alg. 1's order on ties; Alg. 1 above
// kCostPlanMax patterns.  Same outputs as plan_bgp.
int plan_bgp_cost(const gsmat_pattern *pats, int n, const int64_t *keys, const gsmat_pred_stats *stats,
                  int32_t *order, int32_t *kinds, double *est);

// Shape checks shared by gsmat_plan and gsmat_query.
int validate_bgp(const gsmat_pattern *pats, int n_pats, int n_vars);

}  // namespace gs
