"""Oracle for the SM-based BGP join -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  It shares no code with the CUDA path
(``paper_1807_07691_b300``) and never imports it.

Contents:

* ``bgp_join.c`` (through ``OracleIndex``): the definition of a BGP's result
  (Sec. 6 evaluation procedure; Sec. 6.1 join without accumulation),
  evaluated as a nested-loop join in input pattern order over the raw triple
  set.
* ``storage``: the per-predicate sparse matrices M_h and the auxiliary
  arrays Row/Num/Rpos (Sec. 5.3; Sec. 6.3, auxiliary arrays).
* ``planner``: the greedy connected ordering of Alg. 1 and the accumulated
  intermediate-size estimate of Sec. 6.2 (Prop. 1, Thm. 1, Thm. 2).

Parity status: the join and the storage are pinned (paper worked examples,
brute force, invariants; the matrices, their row arrays on both sides and
the row statistics by the D_G example); the planner's order is pinned by the
paper's BGP sequence example; the intermediate-size estimate (a stated
reading, the paper gives only bounds) is pinned by hand-costed cases of
every step kind on D_G's statistics and by the Thm. 1 upper bound.
"""

from .join import OracleIndex, oracle_query, OracleError
from . import storage, planner

__all__ = ["OracleIndex", "oracle_query", "OracleError", "storage", "planner"]
