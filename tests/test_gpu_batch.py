"""Batched evaluation (one persistent kernel for many BGPs) against the
oracle and the plain path, bit-exact (GPU)."""

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import random_bgp

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


def _mixed_bgps(t, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        pats, V = random_bgp(rng, t, n_vars_max=4, n_pats_max=4, p_const=0.45)
        out.append((pats, V))
    return out


def _check_all(B, items, ix):
    for i, (pats, V) in enumerate(items):
        want = ix.query(pats, V, row_limit=20_000_000)
        got = B.to_numpy(i)
        assert got.shape == want.shape, (i, pats)
        assert np.array_equal(got, want), (i, pats)


def test_batch_tiny_workload_and_random_bgps(gs, tiny):
    t, ix, S, qs = tiny
    items = [(q.patterns, q.n_vars) for q in qs] + _mixed_bgps(t, 150, 1)
    # keep the random ones small enough for the oracle
    items = [it for it in items if _small(ix, it)]
    B = gs.Batch(S, [p for p, _ in items], n_vars_list=[v for _, v in items]).execute()
    _check_all(B, items, ix)
    st = B.stats()
    assert st["n_queries"] == len(items)
    assert st["n_in_kernel"] + st["n_reordered"] + st["n_fallback"] == len(items)
    assert st["n_in_kernel"] > 0


def _small(ix, item):
    try:
        ix.query(item[0], item[1], row_limit=2_000_000)
        return True
    except oracle.OracleError:
        return False


def test_batch_edge_cases(gs):
    t = np.array([(1, 7, 2), (2, 7, 3), (3, 7, 3), (2, 8, 1)], dtype=np.int32)
    ix = oracle.OracleIndex(t)
    S = gs.Store(t)
    items = [
        ([(0, 7, 0, 1, 1)], 1),
        ([(1, 7, 2, 0, 0), (0, 7, 1, 1, 1)], 2),
        ([(1, 7, 3, 0, 0), (0, 7, 1, 1, 1)], 2),
        ([(0, 99, 1, 1, 1)], 2),
        ([(0, 7, 1, 1, 1), (2, 8, 3, 1, 1)], 4),
        ([(1, 7, 2, 0, 0)], 0),
        ([(1, 7, 9, 0, 0)], 0),
        ([(0, 7, 1, 1, 1), (0, 7, 1, 1, 1)], 2),
        ([(0, 7, 1, 1, 1), (1, 7, 1, 1, 1)], 2),
        ([(2, 7, 0, 0, 1), (0, 7, 1, 1, 1)], 2),
        ([(0, 7, 3, 1, 0)], 1),
        ([(5000, 7, 0, 0, 1)], 1),
        ([(0, 7, 1, 1, 1), (1, 8, 0, 1, 1), (0, 7, 2, 1, 1)], 3),
    ]
    for use_graph in (1, 0):
        B = gs.Batch(S, [p for p, _ in items], n_vars_list=[v for _, v in items],
                     config={"use_graph": use_graph}).execute()
        _check_all(B, items, ix)


def test_batch_overflow_and_reorder_paths(gs, tiny):
    t, ix, S, qs = tiny
    items = [(q.patterns, q.n_vars) for q in qs]
    # a tiny row cap sends every large query to the plain path
    B = gs.Batch(S, [p for p, _ in items], n_vars_list=[v for _, v in items],
                 config={"max_rows": 100}).execute()
    _check_all(B, items, ix)
    paths = [B.result(i)[2] for i in range(len(items))]
    assert 1 in paths
    # a small arena does the same through the allocator
    B = gs.Batch(S, [p for p, _ in items], n_vars_list=[v for _, v in items],
                 config={"arena_bytes": 1 << 20}).execute()
    _check_all(B, items, ix)
    # results above the shared-memory sort size take the multi-CTA reorder
    B = gs.Batch(S, [p for p, _ in items], n_vars_list=[v for _, v in items]).execute()
    paths = [B.result(i)[2] for i in range(len(items))]
    assert 2 in paths or all(B.result(i)[0] <= 2048 for i in range(len(items)))


def test_batch_graph_replay_identical(gs, tiny):
    t, ix, S, qs = tiny
    items = [(q.patterns, q.n_vars) for q in qs] + _mixed_bgps(t, 40, 9)
    items = [it for it in items if _small(ix, it)]
    B = gs.Batch(S, [p for p, _ in items], n_vars_list=[v for _, v in items])
    B.execute()
    first = [B.to_numpy(i) for i in range(len(items))]
    for _ in range(2):
        B.execute()
        for i in range(len(items)):
            assert np.array_equal(B.to_numpy(i), first[i])


def test_batch_compact_results_rerun(gs, tiny):
    t, ix, S, qs = tiny
    B = gs.Batch(S, qs, config={"compact_results": 1})
    for _ in range(2):
        B.execute()
        for i, q in enumerate(qs):
            assert np.array_equal(B.to_numpy(i), ix.query(q))


def test_batch_autotune(gs, tiny):
    t, ix, S, qs = tiny
    cfg = gs.batch_autotune(S, qs)
    assert cfg["block"] in (128, 256, 512) and cfg["ctas_per_sm"] in (1, 2, 4, 8)
    assert cfg["block"] * cfg["ctas_per_sm"] <= 2048 and cfg["expand_slots"] in (1, 4)
    B = gs.Batch(S, qs, config=cfg).execute()
    for i, q in enumerate(qs):
        assert np.array_equal(B.to_numpy(i), ix.query(q))


def test_batch_cost_plan(gs, tiny):
    t, ix, S, qs = tiny
    items = [(q.patterns, q.n_vars) for q in qs] + _mixed_bgps(t, 80, 21)
    items = [it for it in items if _small(ix, it)]
    B = gs.Batch(S, [p for p, _ in items], n_vars_list=[v for _, v in items], config={"plan_cost": 1}).execute()
    _check_all(B, items, ix)
    # a row cap that sends the large ones to the plain path, planned the same way
    B = gs.Batch(S, [p for p, _ in items], n_vars_list=[v for _, v in items],
                 config={"plan_cost": 1, "max_rows": 100}).execute()
    _check_all(B, items, ix)
    with pytest.raises(gs.GsmatError) as e:
        gs.Batch(S, qs, config={"plan_cost": 2})
    assert e.value.code == 1


@pytest.mark.parametrize("reorder_mode,plan_cost", [(0, 0), (1, 0), (2, 0), (0, 1)])
def test_batched_mix_on_medium_matches_plain_path(gs, reorder_mode, plan_cost):
    import torch

    t = synth.make_graph("medium")
    qs = synth.make_batched_queries(512)
    S = gs.Store(torch.from_numpy(np.array(t, copy=True)).cuda())
    B = gs.Batch(S, qs, config={"reorder_mode": reorder_mode, "plan_cost": plan_cost}).execute()
    st = B.stats()
    assert st["n_in_kernel"] > 0.5 * len(qs) and st["n_reordered"] > 0
    for i, q in enumerate(qs):
        a = B.to_numpy(i)
        b = S.query(q).to_numpy()
        assert a.shape == b.shape and np.array_equal(a, b), q.name


def test_whole_batched_mix_matches_plain_path_and_oracle(gs):
    """All 4096 queries of the batched mix (medium graph) in one batch: every
    result equals the plain path's; every 8th also equals the oracle's rows;
    the mix's cycles run as intersect-expand steps inside the kernel."""
    import torch

    t = synth.make_graph("medium")
    qs = synth.make_batched_queries(4096)
    S = gs.Store(torch.from_numpy(np.array(t, copy=True)).cuda())
    B = gs.Batch(S, qs).execute()
    st = B.stats()
    assert st["n_queries"] == 4096 and st["n_intersect"] > 0
    ix = oracle.OracleIndex(t)
    n_oracle = 0
    for i, q in enumerate(qs):
        a = B.to_numpy(i)
        b = S.query(q).to_numpy()
        assert a.shape == b.shape and np.array_equal(a, b), q.name
        if i % 8 == 0:
            try:
                want = ix.query(q, row_limit=20_000_000)
            except oracle.OracleError:
                continue
            assert np.array_equal(a, want), q.name
            n_oracle += 1
    assert n_oracle >= 480


@pytest.mark.parametrize("block,expand_slots", [(128, 4), (512, 4), (256, 1)])
def test_batch_expand_tile_shapes(gs, tiny, block, expand_slots):
    """Both expand tile shapes the autotuner chooses between give the
    oracle's rows, with every block size."""
    t, ix, S, qs = tiny
    items = [(q.patterns, q.n_vars) for q in qs] + _mixed_bgps(t, 60, 31 + block + expand_slots)
    items = [it for it in items if _small(ix, it)]
    B = gs.Batch(S, [p for p, _ in items], n_vars_list=[v for _, v in items],
                 config={"block": block, "expand_slots": expand_slots}).execute()
    _check_all(B, items, ix)
    with pytest.raises(gs.GsmatError):
        gs.Batch(S, qs, config={"expand_slots": 3})
