"""BGP evaluation on the GPU against the oracle, bit-exact (GPU)."""

import numpy as np
import pytest

import oracle
import oracle.planner as oplan
import synth
from oracle import storage
from tests.helpers import golden, is_sorted_unique, random_bgp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch

    torch.cuda.init()
    import paper_1807_07691_b300 as g

    return g


@pytest.fixture(scope="module")
def tiny(gs):
    t = synth.make_graph("tiny")
    return t, oracle.OracleIndex(t), gs.Store(t), synth.make_queries("tiny", t)


def test_dg_example(gs):
    g = golden("dg_example.json")
    S = gs.Store(np.array(g["cube_spo"], dtype=np.int32))
    T = S.query(g["query"], 4)
    assert T.to_numpy().tolist() == g["answer_xyzw"]
    st = T.stats()
    assert st["order"] == g["plan_order"]
    # one pattern per step (Alg. 2 as printed) gives the paper's intermediates
    U = S.query(g["query"], 4, flags=gs.NO_INTERSECT)
    assert U.stats()["rows"] == g["plan_step_rows"]
    assert U.to_numpy().tolist() == g["answer_xyzw"]
    # by default the third step's expand is fused with the fourth's filter
    assert st["kind"][2:] == [4, 5] and st["rows"][2:] == [1, 1]
    # paper's column order (X, W, Z, Y) = plan order
    P = S.query(g["query"], 4, flags=gs.PLAN_ORDER)
    assert P.col_vars == [0, 3, 2, 1]
    assert P.to_numpy().tolist() == [g["answer_XWZY"]]


def test_tiny_workload_bit_exact(gs, tiny):
    t, ix, S, qs = tiny
    for q in qs:
        want = ix.query(q)
        got = S.query(q).to_numpy()
        assert got.shape == want.shape, q.name
        assert np.array_equal(got, want), q.name


def test_tiny_workload_any_pattern_order(gs, tiny):
    t, ix, S, qs = tiny
    rng = np.random.default_rng(11)
    for q in qs:
        want = ix.query(q)
        for _ in range(2):
            got = S.query(q.permuted(rng.permutation(len(q.patterns)))).to_numpy()
            assert np.array_equal(got, want), q.name


def test_tiny_plan_order_and_count_only(gs, tiny):
    t, ix, S, qs = tiny
    for q in qs:
        want = ix.query(q)
        P = S.query(q, flags=gs.PLAN_ORDER)
        cv = P.col_vars
        got = P.to_numpy()
        assert is_sorted_unique(got)
        ref = want[:, cv]
        ref = ref[np.lexsort(ref.T[::-1])] if len(ref) else ref
        assert np.array_equal(got, ref), q.name
        C = S.query(q, flags=gs.COUNT_ONLY)
        assert C.shape == (want.shape[0], 0)


def test_tiny_rerun_is_identical(gs, tiny):
    t, ix, S, qs = tiny
    for q in qs[:4]:
        a = S.query(q).to_numpy()
        b = S.query(q).to_numpy()
        assert np.array_equal(a, b)


def test_async_copy_on_another_stream(gs, tiny):
    import torch

    t, ix, S, qs = tiny
    side = torch.cuda.Stream()
    held, outs = [], []
    for q in qs:
        T = S.query(q)
        rows, cols = T.shape
        h = torch.empty(max(1, rows * cols), dtype=torch.int32).pin_memory()
        T.copy_to(h, stream=side, sync=False)
        held.append(T)
        outs.append((h, rows, cols))
    side.synchronize()
    for q, T, (h, rows, cols) in zip(qs, held, outs):
        got = h[: rows * cols].numpy().reshape(rows, cols)
        assert np.array_equal(got, ix.query(q)), q.name
        T.free()


@pytest.mark.parametrize("seed", range(60))
def test_random_bgps_small_graphs(gs, seed):
    rng = np.random.default_rng(1000 + seed)
    t = synth.small_random_graph(int(rng.integers(3, 12)), 3, int(rng.integers(1, 80)), seed=seed,
                                 pred_ids=np.array([3, 77, 123456]))
    pats, V = random_bgp(rng, t, n_vars_max=5, n_pats_max=6)
    want = oracle.oracle_query(t, pats, V)
    S = gs.Store(t)
    got = S.query(pats, V).to_numpy()
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def test_edge_cases(gs):
    t = np.array([(1, 7, 2), (2, 7, 3), (3, 7, 3), (2, 8, 1)], dtype=np.int32)
    ix = oracle.OracleIndex(t)
    S = gs.Store(t)
    cases = [
        ([(0, 7, 0, 1, 1)], 1),                        # ?x p ?x
        ([(1, 7, 2, 0, 0), (0, 7, 1, 1, 1)], 2),       # constant pattern present
        ([(1, 7, 3, 0, 0), (0, 7, 1, 1, 1)], 2),       # constant pattern absent
        ([(0, 99, 1, 1, 1)], 2),                       # absent predicate
        ([(0, 7, 1, 1, 1), (2, 8, 3, 1, 1)], 4),       # Cartesian product
        ([(1, 7, 2, 0, 0)], 0),                        # no variables
        ([(1, 7, 9, 0, 0)], 0),
        ([(0, 7, 1, 1, 1), (0, 7, 1, 1, 1)], 2),       # duplicate pattern
        ([(0, 7, 1, 1, 1), (1, 7, 1, 1, 1)], 2),       # repeated var after binding
        ([(2, 7, 0, 0, 1), (0, 7, 1, 1, 1)], 2),       # constant subject
        ([(0, 7, 3, 1, 0)], 1),                        # constant object
        ([(5000, 7, 0, 0, 1)], 1),                     # constant absent from the store
    ]
    for pats, V in cases:
        want = ix.query(pats, V)
        got = S.query(pats, V).to_numpy()
        assert got.shape == want.shape, pats
        assert np.array_equal(got, want), pats
    with pytest.raises(gs.GsmatError) as e:
        S.query(np.array([[0, 0, 1, 1, 1, 1]]), 2)
    assert e.value.code == 2
    with pytest.raises(gs.GsmatError) as e:
        S.query([(0, 7, 1, 1, 1)], 3)
    assert e.value.code == 1


def test_empty_store_query(gs):
    S = gs.Store(np.zeros((0, 3), np.int32))
    T = S.query([(0, 7, 1, 1, 1)], 2)
    assert T.shape == (0, 2)


def test_query_on_torch_stream(gs, tiny):
    import torch

    t, ix, S, qs = tiny
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got = S.query(qs[0], stream=s).to_torch(stream=s)
    s.synchronize()
    assert np.array_equal(got.cpu().numpy(), ix.query(qs[0]))


def test_torch_allocator_hook(gs, tiny):
    t, ix, S, qs = tiny
    gs.use_torch_allocator(True)
    try:
        S2 = gs.Store(t)
        for q in qs[:3]:
            assert np.array_equal(S2.query(q).to_numpy(), ix.query(q))
        del S2
    finally:
        gs.use_torch_allocator(False)


def _cyclic_bgps(t, rng, n):
    """Triangles and 4-cycles over the graph's predicates, some anchored."""
    preds = np.unique(t[:, 1])
    ents = np.unique(t[:, [0, 2]])
    out = []
    for _ in range(n):
        L = int(rng.integers(3, 5))
        pats = []
        for h in range(L):
            a, b = h, (h + 1) % L
            if rng.random() < 0.5:
                a, b = b, a
            pats.append((a, int(rng.choice(preds)), b, True, True))
        if rng.random() < 0.4:  # anchor one variable
            c = int(rng.choice(ents))
            pats = [(c if (sv and s == 0) else s, p, c if (ov and o == 0) else o, sv and s != 0, ov and o != 0)
                    for (s, p, o, sv, ov) in pats]
            remap = {}
            pats = [((remap.setdefault(s, len(remap)) if sv else s), p, (remap.setdefault(o, len(remap)) if ov else o),
                     sv, ov) for (s, p, o, sv, ov) in pats]
            out.append((pats, len(remap)))
        else:
            out.append((pats, L))
    return out


def test_cycles_use_intersect_expand(gs, tiny):
    t, ix, S, qs = tiny
    tri = [q for q in qs if q.shape == "cycle"][0]
    T = S.query(tri)
    assert np.array_equal(T.to_numpy(), ix.query(tri))
    kinds = T.stats()["kind"]
    assert 4 in kinds and 5 in kinds  # GSMAT_STEP_INTERSECT, GSMAT_STEP_FUSED
    rng = np.random.default_rng(77)
    n_isect = 0
    for pats, V in _cyclic_bgps(t, rng, 40):
        want = ix.query(pats, V, row_limit=20_000_000)
        T = S.query(pats, V)
        assert np.array_equal(T.to_numpy(), want), pats
        assert S.query(pats, V, flags=gs.COUNT_ONLY).shape[0] == want.shape[0]
        n_isect += 4 in T.stats()["kind"]
    assert n_isect > 10


def _plan_inputs(t, pats):
    """Per-pattern keys and predicate statistics as the query computes them:
    nnz for a pattern without constants, the constant's row size otherwise
    (the smaller row with two constants), zeros for an absent predicate."""
    u = storage.unique_triples(t).astype(np.int64)
    st = storage.statistics(t)
    keys, stats = [], []
    for (s, p, o, sv, ov) in [tuple(x[:5]) for x in pats]:
        if p not in st:
            keys.append(0)
            stats.append(dict(nnz=0, nr_s=0, nr_o=0))
            continue
        stats.append(st[p])
        rs = int(np.sum((u[:, 1] == p) & (u[:, 0] == s))) if not sv else None
        ro = int(np.sum((u[:, 1] == p) & (u[:, 2] == o))) if not ov else None
        if rs is not None and ro is not None:
            keys.append(min(rs, ro))
        elif rs is not None:
            keys.append(rs)
        elif ro is not None:
            keys.append(ro)
        else:
            keys.append(st[p]["nnz"])
    return keys, stats


def test_cost_plan_same_relation_and_plan(gs, tiny):
    """GSMAT_PLAN_COST: the same relation as the oracle's, by the plan that
    gsmat_plan_cost gives for the store's statistics, never estimated to cost
    more than Alg. 1's."""
    t, ix, S, qs = tiny
    rng = np.random.default_rng(5)
    items = [(q.patterns, q.n_vars) for q in qs]
    while len(items) < 60:
        pats, V = random_bgp(rng, t, n_vars_max=5, n_pats_max=6, p_const=0.3)
        try:
            ix.query(pats, V, row_limit=2_000_000)
        except oracle.OracleError:
            continue
        items.append((pats, V))
    changed = 0
    for pats, V in items:
        want = ix.query(pats, V)
        T = S.query(pats, V, flags=gs.PLAN_COST)
        assert np.array_equal(T.to_numpy(), want), pats
        st = T.stats()
        keys, stats = _plan_inputs(t, pats)
        if all(s["nnz"] > 0 for s in stats):  # (an absent predicate: empty, whatever the plan)
            order, kinds, est = gs.plan(pats, keys, stats, n_vars=V, cost=True)
            assert st["order"] == order == oplan.cost_plan_order(pats, keys, stats)
        g = S.query(pats, V).stats()
        assert st["est_cost"] <= g["est_cost"]
        changed += st["order"] != g["order"]
        assert S.query(pats, V, flags=gs.PLAN_COST | gs.COUNT_ONLY).shape == (want.shape[0], 0)
        P = S.query(pats, V, flags=gs.PLAN_COST | gs.PLAN_ORDER)
        ref = want[:, P.col_vars]
        ref = ref[np.lexsort(ref.T[::-1])] if len(ref) else ref
        assert np.array_equal(P.to_numpy(), ref)
    assert changed > 0


@pytest.mark.parametrize("seed", range(20))
def test_cost_plan_random_small_graphs(gs, seed):
    rng = np.random.default_rng(5000 + seed)
    t = synth.small_random_graph(int(rng.integers(3, 12)), 3, int(rng.integers(1, 80)), seed=seed,
                                 pred_ids=np.array([3, 77, 123456]))
    pats, V = random_bgp(rng, t, n_vars_max=5, n_pats_max=7)
    want = oracle.oracle_query(t, pats, V)
    got = gs.Store(t).query(pats, V, flags=gs.PLAN_COST).to_numpy()
    assert got.shape == want.shape and np.array_equal(got, want)


@pytest.mark.parametrize("expand_items,short_row", [(512, 1), (1024, 16), (4096, 256), (8192, 4096)])
def test_tile_shapes_leave_results_unchanged(gs, tiny, expand_items, short_row):
    """Every tile shape the tuner may pick gives the oracle's rows (the
    tiny workload, random BGPs, the cycles' filters)."""
    t, ix, S, qs = tiny
    S.set_tiles(expand_items, short_row)
    try:
        assert S.tiles() == {"expand_items": expand_items, "short_row": short_row}
        for q in qs:
            assert np.array_equal(S.query(q).to_numpy(), ix.query(q)), q.name
        rng = np.random.default_rng(expand_items + short_row)
        for pats, V in _cyclic_bgps(t, rng, 10):
            want = ix.query(pats, V, row_limit=20_000_000)
            assert np.array_equal(S.query(pats, V).to_numpy(), want)
    finally:
        S.set_tiles()


def test_store_tune_keeps_the_fastest_shape(gs, tiny):
    t, ix, S, qs = tiny
    with pytest.raises(gs.GsmatError):
        S.set_tiles(3000, 64)
    with pytest.raises(gs.GsmatError):
        S.set_tiles(2048, 0)
    best = S.tune(qs)
    assert best["expand_items"] in (512, 1024, 2048, 4096, 8192) and best["short_row"] in (16, 64, 256)
    assert S.tiles() == best
    for q in qs:
        assert np.array_equal(S.query(q).to_numpy(), ix.query(q)), q.name
    S.set_tiles()
