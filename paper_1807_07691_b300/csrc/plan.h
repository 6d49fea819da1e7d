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

// Shape checks shared by gsmat_plan and gsmat_query.
int validate_bgp(const gsmat_pattern *pats, int n_pats, int n_vars);

}  // namespace gs
