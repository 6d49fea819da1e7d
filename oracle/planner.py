"""Query planner, restated plainly -- TEST INFRASTRUCTURE ONLY.

Alg. 1 ("Query Plan Generated", Sec. 6.2.2) orders a BGP's patterns by a
"connected minimal upper bound": sort the patterns by their predicate
statistic, start from the smallest, then repeatedly take, in sorted order,
the first remaining pattern that shares a node with the patterns taken so
far (Sec. 6.2.1, steps 1-4).

Readings (the printed algorithm resets its index every iteration and removes
a pattern in both branches, so the prose of Sec. 6.2.1 is followed):

* nodes shared means shared *variables*; constants do not connect patterns;
* the sort is stable on the input position, so equal statistics keep input
  order (this reproduces the paper's BGP-sequence example);
* a pattern's statistic is m = nnz(M_p), except that a pattern with a
  constant end uses the exact number of entries of that constant's row
  (with two constant ends, the smaller of the two rows);
* when no remaining pattern shares a variable (a disconnected BGP), the
  smallest remaining one is taken, which is a Cartesian product (Sec. 6.2.1
  "avoiding the Cartesian product" can only be met for connected BGPs).

Intermediate-size estimate (Sec. 6.2.1, Prop. 1 and Thm. 1-2 bound the
accumulated number of intermediate results; the paper gives no estimator,
so the formula is a stated reading; the restatement is pinned by
hand-costed cases of every step kind on the paper's D_G statistics and by
the Thm. 1 upper bound): starting from 1 (the empty assignment), each step
multiplies the running estimate by
  CROSS   (no end bound)              key of the pattern
  EXPAND  from a constant end         key (the constant's row size)
  EXPAND  from a bound variable end   nnz / (non-zero rows on that side)
  FILTER  (both ends bound/constant)  min(1, nnz / (nr_s * nr_o))
and the cost is the sum of the running estimates over all steps.

Cost-based variant (the planner that Thm. 2 motivates; Alg. 1 only
approaches its minimum greedily): over all *connected* orders of a BGP of at
most 8 patterns -- orders in which every step after the first takes a
pattern sharing a variable with the patterns taken so far, unless no
remaining pattern does -- take one of least cost.  Readings: the cost is
accumulated step by step in fp64 (the argmin is a decision taken in
floating point, so the summation order is fixed); among equal costs the
order that comes first when orders are compared as sequences of positions
in the stable key order wins (Alg. 1's order is the first connected order
in that comparison, so it wins any tie it is part of); above 8 patterns the
variant is Alg. 1.  Written here as the definition: every permutation,
filtered, costed, first minimum.
"""

from __future__ import annotations

import itertools

STEP_CROSS = 0
STEP_EXPAND_S = 1  # subject end known, object end a new variable (CSR side)
STEP_EXPAND_O = 2  # object end known, subject end a new variable (CSC side)
STEP_FILTER = 3


def pattern_vars(pat) -> set:
    s, p, o, sv, ov = pat[:5]
    vs = set()
    if sv:
        vs.add(int(s))
    if ov:
        vs.add(int(o))
    return vs


def plan_order(patterns, keys) -> list:
    """Alg. 1 with the readings above; returns pattern indices in plan order."""
    n = len(patterns)
    L = sorted(range(n), key=lambda i: (keys[i], i))
    Q = [L.pop(0)]
    N = set(pattern_vars(patterns[Q[0]]))
    while L:
        pick = None
        for i in L:
            if pattern_vars(patterns[i]) & N:
                pick = i
                break
        if pick is None:
            pick = L[0]
        L.remove(pick)
        Q.append(pick)
        N |= pattern_vars(patterns[pick])
    return Q


def classify(pat, bound: set) -> int:
    s, p, o, sv, ov = pat[:5]
    s_known = (not sv) or (int(s) in bound)
    o_known = (not ov) or (int(o) in bound)
    if s_known and o_known:
        return STEP_FILTER
    if s_known:
        return STEP_EXPAND_S
    if o_known:
        return STEP_EXPAND_O
    return STEP_CROSS


def estimate(patterns, order, keys, stats) -> tuple:
    """Running estimates per step and their sum.  ``stats[i]`` holds nnz,
    nr_s, nr_o of pattern i's predicate (zeros when absent)."""
    bound: set = set()
    est = 1.0
    per_step = []
    kinds = []
    for i in order:
        pat = patterns[i]
        kind = classify(pat, bound)
        st = stats[i]
        nnz, nr_s, nr_o = float(st["nnz"]), float(st["nr_s"]), float(st["nr_o"])
        s, p, o, sv, ov = pat[:5]
        if kind == STEP_CROSS:
            f = float(keys[i])
        elif kind == STEP_FILTER:
            f = min(1.0, nnz / (nr_s * nr_o)) if nr_s > 0 and nr_o > 0 else 0.0
        elif kind == STEP_EXPAND_S:
            if not sv:
                f = float(keys[i])
            else:
                f = nnz / nr_s if nr_s > 0 else 0.0
        else:  # STEP_EXPAND_O
            if not ov:
                f = float(keys[i])
            else:
                f = nnz / nr_o if nr_o > 0 else 0.0
        est = est * f
        per_step.append(est)
        kinds.append(kind)
        bound |= pattern_vars(pat)
    return per_step, sum(per_step), kinds


def is_connected_order(patterns, order) -> bool:
    """Every step shares a variable with the steps before it, unless no
    remaining pattern does (then a Cartesian product is unavoidable)."""
    seen = set(pattern_vars(patterns[order[0]]))
    for k in range(1, len(order)):
        vs = pattern_vars(patterns[order[k]])
        if not (vs & seen):
            rest = order[k:]
            if any(pattern_vars(patterns[j]) & seen for j in rest):
                return False
        seen |= vs
    return True


def order_cost(patterns, order, keys, stats) -> float:
    """Sum of the running estimates, accumulated in step order in fp64."""
    per_step, _, _ = estimate(patterns, order, keys, stats)
    total = 0.0
    for e in per_step:
        total = total + e
    return total


def cost_plan_order(patterns, keys, stats, max_patterns: int = 8) -> list:
    """Least-cost connected order (see the module docstring); Alg. 1's order
    for BGPs of more than ``max_patterns`` patterns."""
    n = len(patterns)
    if n > max_patterns:
        return plan_order(patterns, keys)
    L = sorted(range(n), key=lambda i: (keys[i], i))
    best_cost, best = None, None
    for perm in itertools.permutations(L):  # lexicographic in key positions
        if not is_connected_order(patterns, perm):
            continue
        c = order_cost(patterns, perm, keys, stats)
        if best_cost is None or c < best_cost:
            best_cost, best = c, list(perm)
    return best


def upper_bound_sum(sizes) -> int:
    """Thm. 1's upper bound on the accumulated intermediate results of
    joining relations of the given sizes in the given order:
    |R1||R2| + |R1||R2||R3| + ... + |R1|...|Rn|."""
    total = 0
    prod = 1
    for i, r in enumerate(sizes):
        prod *= int(r)
        if i >= 1:
            total += prod
    return total
