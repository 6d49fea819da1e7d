"""The product step: the plan's last steps whose lists depend only on the
table before them (EXPAND from an earlier variable or from a constant,
CROSS) run as one Cartesian product per input row, nested by variable id
(GPU).

Every result is compared with the oracle and with the same query run one
pattern per step (GSMAT_NO_INTERSECT, which also turns the product off).
Integer results: tolerance zero."""

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import random_bgp

pytestmark = pytest.mark.gpu

PRODUCT = 6  # GSMAT_STEP_PRODUCT


@pytest.fixture(scope="module")
def gs():
    import torch

    torch.cuda.init()
    import paper_1807_07691_b300 as g

    return g


@pytest.fixture(scope="module")
def tiny(gs):
    t = synth.make_graph("tiny")
    return t, oracle.OracleIndex(t), gs.Store(t)


def _check(gs, S, ix, pats, V, expect_product=None, limit=50_000_000):
    want = ix.query(pats, V, row_limit=limit)
    T = S.query(pats, V)
    got = T.to_numpy()
    assert got.shape == want.shape and np.array_equal(got, want), pats
    U = S.query(pats, V, flags=gs.NO_INTERSECT)
    assert PRODUCT not in U.stats()["kind"]
    assert np.array_equal(U.to_numpy(), want)
    assert S.query(pats, V, flags=gs.COUNT_ONLY).rows == want.shape[0]
    st = T.stats()
    if expect_product is not None:
        assert (PRODUCT in st["kind"]) == expect_product, (pats, st["kind"])
    return st, want


def _out_rows(t, s):
    """(predicate, object list) of subject s, by predicate."""
    sub = t[t[:, 0] == s]
    by = {}
    for p, o in sub[:, 1:].tolist():
        by.setdefault(p, []).append(o)
    return {p: sorted(v) for p, v in by.items()}


def test_star_around_a_constant_is_one_product_in_variable_order(gs, tiny):
    """c p_i ?v_i: every list is a constant's row, so the whole query is a
    product of fixed lists; the variables are numbered against the plan's
    (row-size) order so that a plain run would have to reorder."""
    t, ix, S = tiny
    rng = np.random.default_rng(3)
    subjects, counts = np.unique(t[:, 0], return_counts=True)
    done = 0
    for s in subjects[np.argsort(-counts)][:200].tolist():
        rows = _out_rows(t, s)
        if len(rows) < 3:
            continue
        preds = sorted(rows, key=lambda p: -len(rows[p]))[:4]  # longest row first: ids against the plan
        pats = [(s, p, v, False, True) for v, p in enumerate(preds)]
        st, want = _check(gs, S, ix, pats, len(preds), expect_product=True)
        assert all(k == PRODUCT for k in st["kind"])
        # exact running products in plan order (rows of the plan's steps)
        lens = [len(rows[preds[i]]) for i in st["order"]]
        assert st["rows"] == list(np.cumprod(lens))
        assert want.shape[0] == int(np.prod([len(rows[p]) for p in preds]))
        # the same with shuffled variable ids
        perm = rng.permutation(len(preds))
        pats2 = [(s, p, int(perm[v]), False, True) for v, p in enumerate(preds)]
        _check(gs, S, ix, pats2, len(preds), expect_product=True)
        done += 1
        if done == 6:
            break
    assert done == 6


def test_star_around_a_variable_runs_the_leaves_as_a_product(gs, tiny):
    """?c bound first (from a constant object), then every other pattern
    expands from ?c: a product per row of ?c."""
    t, ix, S = tiny
    objs, counts = np.unique(t[:, 2], return_counts=True)
    rng = np.random.default_rng(4)
    n_prod = 0
    for o in objs[np.argsort(-counts)][:60].tolist():
        anchor_p = int(t[t[:, 2] == o][0, 1])
        preds = rng.choice(np.unique(t[:, 1]), size=3, replace=False).tolist()
        for order in ([1, 2, 3], [3, 1, 2], [2, 3, 1]):
            pats = [(0, anchor_p, o, True, False)] + [(0, int(p), v, True, True) for p, v in zip(preds, order)]
            st, want = _check(gs, S, ix, pats, 4)
            n_prod += PRODUCT in st["kind"]
    assert n_prod > 0


def test_snowflakes_and_random_bgps(gs, tiny):
    t, ix, S = tiny
    rng = np.random.default_rng(5)
    n_prod = checked = 0
    while checked < 150:
        pats, V = random_bgp(rng, t, n_vars_max=6, n_pats_max=6, p_const=0.3)
        try:
            ix.query(pats, V, row_limit=3_000_000)
        except oracle.OracleError:
            continue
        st, _ = _check(gs, S, ix, pats, V)
        n_prod += PRODUCT in st["kind"]
        checked += 1
    assert n_prod >= 3  # random BGPs seldom end in independent expansions


@pytest.mark.parametrize("seed", range(12))
def test_products_of_whole_matrices_and_empty_lists(gs, seed):
    """Disconnected BGPs (CROSS factors: pairs of a whole matrix), constants
    without a row (an empty list), repeated ids, on small random graphs."""
    rng = np.random.default_rng(900 + seed)
    t = synth.small_random_graph(int(rng.integers(3, 10)), 3, int(rng.integers(1, 60)), seed=seed,
                                 pred_ids=np.array([5, 91, 4000]))
    S = gs.Store(t)
    ix = oracle.OracleIndex(t)
    for _ in range(12):
        pats, V = random_bgp(rng, t, n_vars_max=6, n_pats_max=4, p_const=0.35, p_selfloop=0.0)
        _check(gs, S, ix, pats, V)
    # two and three whole matrices side by side
    for k in (2, 3):
        pats = [(2 * i, [5, 91, 4000][i % 3], 2 * i + 1, True, True) for i in range(k)]
        _check(gs, S, ix, pats, 2 * k)
    # a factor with an absent constant row: empty
    pats = [(0, 5, 1, True, True), (10_000, 91, 2, False, True)]
    st, want = _check(gs, S, ix, pats, 3)
    assert want.shape[0] == 0


def test_product_shards_partition_the_result(gs, tiny):
    t, ix, S = tiny
    subjects, counts = np.unique(t[:, 0], return_counts=True)
    s = int(subjects[np.argmax(counts)])
    rows = _out_rows(t, s)
    preds = sorted(rows, key=lambda p: -len(rows[p]))[:3]
    pats = [(s, p, v, False, True) for v, p in enumerate(preds)]
    want = ix.query(pats, len(preds))
    for n_shards in (2, 3, 5):
        parts = [S.query_shard(pats, k, n_shards, n_vars=len(preds)) for k in range(n_shards)]
        assert sum(p.rows for p in parts) == want.shape[0]
        assert np.array_equal(gs.merge_tables(parts).to_numpy(), want)


def _rows_by(t, side):
    """{(entity, predicate): sorted other ends} for one side (0: by subject)."""
    by = {}
    a, b = (0, 2) if side == 0 else (2, 0)
    for row in t.tolist():
        by.setdefault((row[a], row[1]), []).append(row[b])
    return {k: sorted(v) for k, v in by.items()}


def test_constant_rows_first_then_their_expansions(gs, tiny):
    """Two or three constant rows (c_i p_i ?a_i) and expansions of their
    variables (?a_i q ?x): the constant rows run first as one product in
    variable order, then the expansions as a product per row.  Variable
    ids are shuffled so that the final order differs from the binding
    order in some cases."""
    t, ix, S = tiny
    rng = np.random.default_rng(11)
    by_s = _rows_by(t, 0)
    starts = [(k, v) for k, v in by_s.items() if 2 <= len(v) <= 40]
    preds_of = {}
    for (e, p) in by_s:
        preds_of.setdefault(e, []).append(p)
    hoisted = checked = 0
    while checked < 40:
        n_fix = int(rng.integers(2, 4))
        pick = [starts[i] for i in rng.choice(len(starts), size=n_fix, replace=False)]
        pats, V = [], 0
        fix_vars = []
        for (c, p), _ in pick:
            pats.append((c, p, V, False, True))
            fix_vars.append(V)
            V += 1
        # expansions from the constant rows' variables, by a predicate one of
        # their values has
        for k, ((c, p), objs) in enumerate(pick):
            for _ in range(int(rng.integers(1, 3))):
                o = objs[int(rng.integers(0, len(objs)))]
                if o not in preds_of:
                    continue
                q = preds_of[o][int(rng.integers(0, len(preds_of[o])))]
                pats.append((fix_vars[k], q, V, True, True))
                V += 1
        if len(pats) == n_fix:
            continue
        perm = rng.permutation(V)
        pats = [(int(perm[s]) if sv else s, p, int(perm[o]) if ov else o, sv, ov) for s, p, o, sv, ov in pats]
        try:
            ix.query(pats, V, row_limit=20_000_000)
        except oracle.OracleError:
            continue
        st, want = _check(gs, S, ix, pats, V)
        order = st["order"]
        if all(k == PRODUCT for k in st["kind"][:n_fix]) and sorted(order[:n_fix]) == list(range(n_fix)):
            hoisted += 1
            # the constant rows' product is exact: the running products of their lengths
            lens = [len(pick[i][1]) for i in order[:n_fix]]
            assert st["rows"][:n_fix] == list(np.cumprod(lens))
        checked += 1
    assert hoisted >= 20
