"""Pins of the oracle against what the paper and mathematics fix (CPU only).

Each test names the passage it checks.  The oracle is compared with worked
examples printed in the paper, brute-force enumeration, a matrix-product
closed form and invariants; never with itself.
"""

import itertools

import numpy as np
import pytest

import oracle
import synth
from oracle import planner, storage
from tests.helpers import brute_force, golden, is_sorted_unique, random_bgp, satisfies_all


# --------------------------------------------------------------------------
# Worked example D_G (Sec. 3.1, 5.2, 5.3, 6.3)


def test_dg_answer_is_the_papers_single_row():
    g = golden("dg_example.json")
    ix = oracle.OracleIndex(np.array(g["cube_spo"]))
    rows = ix.query(g["query"], 4)
    assert rows.tolist() == g["answer_xyzw"]
    # the paper prints it over (X, W, Z, Y)
    x, y, z, w = rows[0]
    assert [x, w, z, y] == g["answer_XWZY"]


def test_dg_intermediate_rows_in_paper_plan_order():
    g = golden("dg_example.json")
    ix = oracle.OracleIndex(np.array(g["cube_spo"]))
    q = [g["query"][i] for i in g["plan_order"]]
    rows, steps = ix.query(q, 4, return_steps=True)
    assert steps.tolist() == g["plan_step_rows"]


def test_dg_matrices_and_statistics():
    g = golden("dg_example.json")
    mats = storage.sparse_matrices(np.array(g["cube_spo"]))
    assert {str(k): v.tolist() for k, v in mats.items()} == g["matrices"]
    stats = storage.statistics(np.array(g["cube_spo"]))
    assert [stats[h]["nnz"] for h in (1, 2, 3)] == [3, 4, 2]
    # Sec. 5.3: 9 pairs = 18 units against 7*7*3 = 147 for adjacency storage
    assert sum(2 * s["nnz"] for s in stats.values()) == g["storage_units"]["sm_units"]
    assert len(g["h_so"]) * len(g["h_so"]) * len(g["h_p"]) == g["storage_units"]["adjacency_units"]


def test_dg_auxiliary_arrays():
    g = golden("dg_example.json")
    M1 = storage.sparse_matrices(np.array(g["cube_spo"]))[1]
    assert storage.aux_arrays(M1, 0).tolist() == g["aux_A_X"]
    assert g["aux_B_W_entry"] in storage.aux_arrays(M1, 1).tolist()


def test_dg_csr_by_both_sides():
    """csr_by: the doubly-compressed rows of every M_h (Sec. 5.3) on the
    subject side (CSR) and the object side (CSC), i.e. the Row and Rpos
    arrays of Sec. 6.3 for either join column.  Expected arrays: the printed
    matrices read row by row by hand (fixture)."""
    g = golden("dg_example.json")
    cube = np.array(g["cube_spo"])
    for side, key in (("s", "csr_by_s"), ("o", "csr_by_o")):
        got = storage.csr_by(cube, side)
        assert sorted(got) == [1, 2, 3]
        for h, (rid, ptr, ent) in got.items():
            assert [rid.tolist(), ptr.tolist(), ent.tolist()] == g[key][str(h)], (side, h)
    # (Row, Num, Rpos) of :likes on X as printed: Num = pointer difference,
    # Rpos = pointer + 1
    rid, ptr, _ = storage.csr_by(cube, "s")[1]
    aux = [[int(r), int(ptr[i + 1] - ptr[i]), int(ptr[i]) + 1] for i, r in enumerate(rid)]
    assert aux == g["aux_A_X"]
    # and the entry of :likes on W (object side) that the paper prints
    rid, ptr, _ = storage.csr_by(cube, "o")[1]
    aux_o = [[int(r), int(ptr[i + 1] - ptr[i]), int(ptr[i]) + 1] for i, r in enumerate(rid)]
    assert g["aux_B_W_entry"] in aux_o


def test_dg_statistics_row_counts():
    """statistics: m = nnz (Sec. 5.3) and the distinct subjects and objects
    of each printed matrix (nr_s, nr_o), counted by hand (fixture)."""
    g = golden("dg_example.json")
    stats = storage.statistics(np.array(g["cube_spo"]))
    assert {str(h): [s["nnz"], s["nr_s"], s["nr_o"]] for h, s in stats.items()} == g["stats_nnz_nrs_nro"]


def _dg_stats():
    # (nnz, nr_s, nr_o) of :likes (1), :follows (2), :related (3), as in the fixture
    g = golden("dg_example.json")
    return {int(h): dict(nnz=v[0], nr_s=v[1], nr_o=v[2]) for h, v in g["stats_nnz_nrs_nro"].items()}


def test_estimate_filter_step_hand_costed():
    """The FILTER factor min(1, nnz / (nr_s nr_o)) of the estimate (Sec.
    6.2.1 reading), costed by hand on D_G's statistics:
      ?x :likes ?w . ?x :follows ?w   in that order
      CROSS 3 (m of :likes), then FILTER by :follows: 3 * 4/(3*3) = 4/3;
      cost 3 + 4/3 = 13/3.
      ?x :follows ?w . ?x :related ?w: 4, then 4 * 2/(2*1) = 4; cost 8."""
    st = _dg_stats()
    pats = [(0, 1, 1, 1, 1), (0, 2, 1, 1, 1)]
    per_step, total, kinds = planner.estimate(pats, [0, 1], [3, 4], [st[1], st[2]])
    assert kinds == [planner.STEP_CROSS, planner.STEP_FILTER]
    assert per_step == pytest.approx([3.0, 4.0 / 3.0], rel=1e-15)
    assert total == pytest.approx(13.0 / 3.0, rel=1e-15)
    pats = [(0, 2, 1, 1, 1), (0, 3, 1, 1, 1)]
    per_step, total, kinds = planner.estimate(pats, [0, 1], [4, 2], [st[2], st[3]])
    assert kinds == [planner.STEP_CROSS, planner.STEP_FILTER]
    assert per_step == [4.0, 4.0] and total == 8.0


def test_estimate_constant_anchored_expand_hand_costed():
    """EXPAND from a constant end multiplies by that constant's row size
    (its key); EXPAND from a bound variable by nnz / nr on that side; a
    pattern with a constant end whose other end is bound is a FILTER.  By
    hand on D_G (A = 1, I2 = 3):
      A :follows ?y . ?y :follows ?z . ?z :likes I2
        A's :follows row has 1 entry      -> 1
        * nnz/nr_s of :follows = 4/3      -> 4/3
        * FILTER 3/(2*2) of :likes        -> 1;      cost 1 + 4/3 + 1 = 10/3
      ?x :likes I2 . ?x :follows ?y
        I2's :likes column has 2 entries  -> 2  (object side)
        * 4/3                             -> 8/3;    cost 2 + 8/3 = 14/3"""
    st = _dg_stats()
    pats = [(1, 2, 0, 0, 1), (0, 2, 1, 1, 1), (1, 1, 3, 1, 0)]
    per_step, total, kinds = planner.estimate(pats, [0, 1, 2], [1, 4, 2], [st[2], st[2], st[1]])
    assert kinds == [planner.STEP_EXPAND_S, planner.STEP_EXPAND_S, planner.STEP_FILTER]
    assert per_step == pytest.approx([1.0, 4.0 / 3.0, 1.0], rel=1e-15)
    assert total == pytest.approx(10.0 / 3.0, rel=1e-15)
    pats = [(0, 1, 3, 1, 0), (0, 2, 1, 1, 1)]
    per_step, total, kinds = planner.estimate(pats, [0, 1], [2, 4], [st[1], st[2]])
    assert kinds == [planner.STEP_EXPAND_O, planner.STEP_EXPAND_S]
    assert per_step == pytest.approx([2.0, 8.0 / 3.0], rel=1e-15)
    assert total == pytest.approx(14.0 / 3.0, rel=1e-15)
    # the hand-counted row sizes are the oracle's rows for those constants
    ix = oracle.OracleIndex(np.array(golden("dg_example.json")["cube_spo"]))
    assert ix.query([(1, 2, 0, 0, 1)], 1).shape[0] == 1
    assert ix.query([(0, 1, 3, 1, 0)], 1).shape[0] == 2


def test_dg_first_intermediate_row():
    g = golden("dg_example.json")
    ix = oracle.OracleIndex(np.array(g["cube_spo"]))
    # ?X likes ?W . ?Z likes ?W over variables X=0, W=1, Z=2
    rows = ix.query([(0, 1, 1, 1, 1), (2, 1, 1, 1, 1)], 3)
    assert g["first_C_row_XWZ"] == rows[0].tolist()


def test_dg_plan_order_matches_bgp_sequence():
    g = golden("dg_example.json")
    cube = np.array(g["cube_spo"])
    stats = storage.statistics(cube)
    keys = [stats[p[1]]["nnz"] for p in g["query"]]
    assert planner.plan_order(g["query"], keys) == g["plan_order"]


# --------------------------------------------------------------------------
# Join without accumulation (Sec. 6.1)


def test_spgemm_example_join_keeps_all_columns():
    g = golden("spgemm_example.json")
    L = g["letters"]
    A, B = 10, 11
    trip = [(L[a], A, L[b]) for a, b in g["A"]] + [(L[a], B, L[b]) for a, b in g["B"]]
    rows = oracle.oracle_query(np.array(trip), [(0, A, 1, 1, 1), (1, B, 2, 1, 1)], 3)
    want = sorted([L[a], L[b], L[c]] for a, b, c in g["join_rows"])
    assert rows.tolist() == want
    # accumulated value c_it = 2 appears as two distinct rows (i,k,t), (i,l,t)
    for a, c, v in g["C_product"]:
        n = sum(1 for r in rows.tolist() if r[0] == L[a] and r[2] == L[c])
        assert n == v


def _adj(triples, p, n):
    M = np.zeros((n, n), dtype=np.int64)
    for s, pp, o in np.asarray(triples).tolist():
        if pp == p:
            M[s, o] = 1
    return M


@pytest.mark.parametrize("seed", range(6))
def test_chain_counts_equal_boolean_matrix_product(seed):
    """For ?x p1 ?y . ?y p2 ?z, the number of rows with given (x, z) is
    (A1 A2)[x, z] (Sec. 6.1: the join is the product without accumulation)."""
    n = 9
    t = synth.small_random_graph(n, 3, 60, seed=seed)
    p1, p2 = 0, (seed % 3)
    rows = oracle.oracle_query(t, [(0, p1, 1, 1, 1), (1, p2, 2, 1, 1)], 3)
    C = _adj(t, p1, n) @ _adj(t, p2, n)
    got = np.zeros((n, n), dtype=np.int64)
    for x, y, z in rows.tolist():
        got[x, z] += 1
    assert (got == C).all()


@pytest.mark.parametrize("seed", range(6))
def test_star_counts_equal_degree_products(seed):
    """A constant-free star ?x p_i ?y_i has sum_x prod_i deg_{p_i}(x) rows."""
    n = 10
    t = synth.small_random_graph(n, 3, 80, seed=100 + seed)
    ps = [seed % 3, (seed + 1) % 3, 0]
    rows = oracle.oracle_query(t, [(0, p, i + 1, 1, 1) for i, p in enumerate(ps)], 4)
    deg = [_adj(t, p, n).sum(axis=1) for p in ps]
    assert rows.shape[0] == int(np.prod(deg, axis=0).sum())


# --------------------------------------------------------------------------
# Brute force on tiny graphs


@pytest.mark.parametrize("seed", range(40))
def test_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n_ent = int(rng.integers(3, 9))
    t = synth.small_random_graph(n_ent, 3, int(rng.integers(5, 40)), seed=seed, pred_ids=np.array([5, 9, 1000]))
    pats, V = random_bgp(rng, t, n_vars_max=4, n_pats_max=5)
    want = brute_force(t, pats, V)
    got = oracle.oracle_query(t, pats, V)
    assert got.shape == want.shape
    assert (got == want).all()


def test_duplicate_input_triples_are_one_triple():
    t = np.array([(1, 7, 2), (1, 7, 2), (2, 7, 3), (1, 7, 2)])
    rows = oracle.oracle_query(t, [(0, 7, 1, 1, 1)], 2)
    assert rows.tolist() == [[1, 2], [2, 3]]


def test_edge_cases():
    t = np.array([(1, 7, 2), (2, 7, 3), (3, 7, 3), (2, 8, 1)])
    ix = oracle.OracleIndex(t)
    # repeated variable
    assert ix.query([(0, 7, 0, 1, 1)], 1).tolist() == [[3]]
    # both ends constant: present / absent
    assert ix.query([(1, 7, 2, 0, 0), (0, 7, 1, 1, 1)], 2).shape == (3, 2)
    assert ix.query([(1, 7, 3, 0, 0), (0, 7, 1, 1, 1)], 2).shape == (0, 2)
    # absent predicate: empty, not an error
    assert ix.query([(0, 99, 1, 1, 1)], 2).shape == (0, 2)
    # disconnected: Cartesian product
    assert ix.query([(0, 7, 1, 1, 1), (2, 8, 3, 1, 1)], 4).shape == (3, 4)
    # no variables at all
    assert ix.query([(1, 7, 2, 0, 0)], 0).shape == (1, 0)
    assert ix.query([(1, 7, 9, 0, 0)], 0).shape == (0, 0)
    # variable predicate is unsupported (Sec. 6.3 assumes known predicates)
    with pytest.raises(oracle.OracleError) as e:
        ix.query(np.array([[0, 0, 1, 1, 1, 1]]), 2)
    assert e.value.code == 2
    # a declared variable that no pattern uses is invalid
    with pytest.raises(oracle.OracleError):
        ix.query([(0, 7, 1, 1, 1)], 3)


# --------------------------------------------------------------------------
# Invariants on the tiny workload


@pytest.fixture(scope="module")
def tiny():
    t = synth.make_graph("tiny")
    return t, oracle.OracleIndex(t), synth.make_queries("tiny", t)


def test_tiny_workload_invariants(tiny):
    t, ix, qs = tiny
    for q in qs:
        rows = ix.query(q)
        assert rows.shape[0] > 0, q.name  # drawn from an instance
        assert is_sorted_unique(rows)
        assert satisfies_all(t, q.patterns, rows)


def test_tiny_order_invariance(tiny):
    t, ix, qs = tiny
    rng = np.random.default_rng(3)
    for q in qs[:6]:
        base = ix.query(q)
        perm = rng.permutation(len(q.patterns))
        assert (ix.query(q.permuted(perm)) == base).all()


def test_renaming_invariance(tiny):
    """Applying a bijection to entity ids maps the result by the same
    bijection (the method never interprets ids)."""
    t, ix, qs = tiny
    rng = np.random.default_rng(5)
    E = int(t[:, [0, 2]].max()) + 1
    f = rng.permutation(E).astype(np.int64) + 1000
    t2 = t.astype(np.int64).copy()
    t2[:, 0] = f[t2[:, 0]]
    t2[:, 2] = f[t2[:, 2]]
    ix2 = oracle.OracleIndex(t2)
    for q in qs[:5]:
        q2 = [(s if sv else int(f[s]), p, o if ov else int(f[o]), sv, ov) for (s, p, o, sv, ov) in q.patterns]
        a = ix.query(q)
        b = ix2.query(q2, q.n_vars)
        mapped = f[a.astype(np.int64)]
        mapped = mapped[np.lexsort(mapped.T[::-1])] if mapped.size else mapped
        assert (mapped == b).all()


# --------------------------------------------------------------------------
# Planner and cost bounds (Sec. 6.2)


def test_upper_bound_sum_and_thm2_ascending_minimises():
    assert planner.upper_bound_sum([2, 3, 4]) == 2 * 3 + 2 * 3 * 4
    rng = np.random.default_rng(0)
    for _ in range(30):
        sizes = rng.integers(1, 50, size=int(rng.integers(2, 6))).tolist()
        best = min(planner.upper_bound_sum(p) for p in itertools.permutations(sizes))
        assert planner.upper_bound_sum(sorted(sizes)) == best


def test_thm1_upper_bound_holds_for_oracle_intermediates(tiny):
    t, ix, qs = tiny
    stats = storage.statistics(t)
    for q in qs:
        rows, steps = ix.query(q, return_steps=True)
        sizes = [stats[p[1]]["nnz"] for p in q.patterns]
        assert int(steps[1:].sum()) <= planner.upper_bound_sum(sizes)
        assert int(steps[0]) <= sizes[0]


def _connected(pats):
    seen = set(planner.pattern_vars(pats[0]))
    left = list(pats[1:])
    while left:
        nxt = [p for p in left if planner.pattern_vars(p) & seen]
        if not nxt:
            return False
        for p in nxt:
            seen |= planner.pattern_vars(p)
            left.remove(p)
    return True


def test_plan_never_takes_a_cartesian_step_on_connected_bgps():
    """Sec. 6.2.1 step 3: every pattern after the first shares a variable
    with those taken before it, whenever the BGP allows it."""
    rng = np.random.default_rng(2)
    n_checked = 0
    for _ in range(300):
        n = int(rng.integers(2, 7))
        pats = [(int(rng.integers(4)), 1, int(rng.integers(4)), 1, 1) for _ in range(n)]
        if not _connected(pats):
            continue
        n_checked += 1
        keys = rng.integers(0, 100, size=n).tolist()
        order = planner.plan_order(pats, keys)
        assert sorted(order) == list(range(n))
        seen = set(planner.pattern_vars(pats[order[0]]))
        for i in order[1:]:
            assert planner.pattern_vars(pats[i]) & seen
            seen |= planner.pattern_vars(pats[i])
    assert n_checked > 50


def test_plan_first_pattern_has_smallest_key():
    rng = np.random.default_rng(1)
    for _ in range(50):
        n = int(rng.integers(1, 7))
        pats = [(int(rng.integers(3)), 1, int(rng.integers(3)), 1, 1) for _ in range(n)]
        keys = rng.integers(0, 5, size=n).tolist()
        order = planner.plan_order(pats, keys)
        assert keys[order[0]] == min(keys)
        assert order[0] == keys.index(min(keys))


# --------------------------------------------------------------------------
# Cost-based planner variant (Thm. 2 motivates minimising the accumulated
# estimate; Alg. 1 approaches it greedily)


def _chain_abc():
    # ?x A ?y . ?y B ?z . ?z C ?w -- A is the smallest matrix, but all of its
    # 100 entries point at one object, whose row in B holds 150 entries
    pats = [(0, 1, 1, 1, 1), (1, 2, 2, 1, 1), (2, 3, 3, 1, 1)]
    stats = [dict(nnz=100, nr_s=100, nr_o=1), dict(nnz=150, nr_s=1, nr_o=150), dict(nnz=200, nr_s=200, nr_o=200)]
    keys = [100, 150, 200]
    return pats, keys, stats


def test_cost_plan_worked_chain():
    """Costs written out by hand for every connected order of the chain
    A-B-C (running estimates: CROSS -> key, EXPAND -> nnz / nr of the bound
    side):
      A,B,C: 100, 100*150/1, *200/200        -> 100 + 15000 + 15000 = 30100
      B,A,C: 150, 150*100/1, *200/200        -> 150 + 15000 + 15000 = 30150
      B,C,A: 150, 150*200/200, *100/1        -> 150 + 150 + 15000   = 15300
      C,B,A: 200, 200*150/150, *100/1        -> 200 + 200 + 20000   = 20400
    (A,C,B and C,A,B join two patterns that share nothing while B connects)."""
    pats, keys, stats = _chain_abc()
    assert planner.plan_order(pats, keys) == [0, 1, 2]
    assert planner.order_cost(pats, [0, 1, 2], keys, stats) == 30100.0
    order = planner.cost_plan_order(pats, keys, stats)
    assert order == [1, 2, 0]
    per_step, _, kinds = planner.estimate(pats, order, keys, stats)
    assert per_step == [150.0, 150.0, 15000.0]
    assert kinds == [planner.STEP_CROSS, planner.STEP_EXPAND_S, planner.STEP_EXPAND_O]
    assert planner.order_cost(pats, order, keys, stats) == 15300.0
    assert not planner.is_connected_order(pats, [0, 2, 1])
    assert planner.is_connected_order(pats, [2, 1, 0])


def test_cost_plan_tie_keeps_alg1_order():
    """Two patterns of key 4 (nnz 4 over 2 rows on each side) sharing ?y:
    either order costs 4 + 4*2 = 12, so the stable key order (Alg. 1's) is
    kept; with the keys swapped the other order is Alg. 1's and is kept."""
    pats = [(0, 1, 1, 1, 1), (1, 2, 2, 1, 1)]
    st = [dict(nnz=4, nr_s=2, nr_o=2)] * 2
    assert planner.order_cost(pats, [0, 1], [4, 4], st) == planner.order_cost(pats, [1, 0], [4, 4], st) == 12.0
    assert planner.cost_plan_order(pats, [4, 4], st) == [0, 1]
    assert planner.cost_plan_order(pats, [5, 4], st) == [1, 0] == planner.plan_order(pats, [5, 4])


def test_cost_plan_disconnected_bgp_takes_a_cartesian_step():
    # {?x A ?y} and {?z B ?w} share nothing: both orders are connected in the
    # sense above; costs 3 + 3*7 = 24 (A first) and 7 + 7*3 = 28 (B first)
    pats = [(0, 1, 1, 1, 1), (2, 2, 3, 1, 1)]
    st = [dict(nnz=3, nr_s=3, nr_o=3), dict(nnz=7, nr_s=7, nr_o=7)]
    assert planner.is_connected_order(pats, [1, 0])
    assert planner.cost_plan_order(pats, [3, 7], st) == [0, 1]
    assert planner.order_cost(pats, [0, 1], [3, 7], st) == 24.0


def test_cost_plan_never_costs_more_than_alg1_and_stays_connected():
    rng = np.random.default_rng(11)
    improved = 0
    for _ in range(120):
        n = int(rng.integers(1, 7))
        pats = [(int(rng.integers(4)), int(rng.integers(3)), int(rng.integers(4)), 1, int(rng.random() < 0.9))
                for _ in range(n)]
        keys = rng.integers(1, 1000, size=n).tolist()
        stats = [dict(nnz=int(rng.integers(1, 5000)), nr_s=int(rng.integers(1, 100)), nr_o=int(rng.integers(1, 100)))
                 for _ in range(n)]
        g = planner.plan_order(pats, keys)
        c = planner.cost_plan_order(pats, keys, stats)
        assert sorted(c) == list(range(n))
        assert planner.is_connected_order(pats, c) and planner.is_connected_order(pats, g)
        gc, cc = planner.order_cost(pats, g, keys, stats), planner.order_cost(pats, c, keys, stats)
        assert cc <= gc
        improved += cc < gc
    assert improved > 10


def test_cost_plan_above_eight_patterns_is_alg1():
    pats = [(i, 1, i + 1, 1, 1) for i in range(9)]
    keys = list(range(9, 0, -1))
    st = [dict(nnz=10, nr_s=5, nr_o=5)] * 9
    assert planner.cost_plan_order(pats, keys, st) == planner.plan_order(pats, keys)


def test_cost_plan_result_is_the_same_relation(tiny):
    """The plan changes the order of the joins, never the relation (Sec. 6.1):
    the oracle evaluated in the cost plan's order gives the same rows."""
    t, ix, qs = tiny
    st = storage.statistics(t)
    for q in qs:
        stats = [st[p[1]] for p in q.patterns]
        keys = [s["nnz"] for s in stats]
        order = planner.cost_plan_order(q.patterns, keys, stats)
        want = ix.query(q.patterns, q.n_vars)
        got = ix.query([q.patterns[i] for i in order], q.n_vars)
        assert np.array_equal(got, want)


def test_large_served_mix_counts_match_the_oracle():
    # the anchored sampler's exact counts (stars, chains) on the tiny graph
    t = synth.make_graph("tiny")
    qs = synth.make_large_served_queries(t, n_queries=36, n_entities=10_000, limit=2e5)
    ix = oracle.OracleIndex(t)
    shapes = {q.shape for q in qs}
    assert shapes == {"star", "chain", "snowflake"}
    for q in qs:
        assert 2 <= len(q.patterns) <= 8
        got = ix.query(q, row_limit=5_000_000)
        assert got.shape[0] <= q.bound + 1e-6, q.name
        if q.count is not None:
            assert got.shape[0] == int(q.count), q.name
