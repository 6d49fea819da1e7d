"""Device store builder against the oracle's per-predicate matrices (GPU)."""

import numpy as np
import pytest

import synth
from oracle import storage
from tests.helpers import golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch

    torch.cuda.init()
    import paper_1807_07691_b300 as g

    return g


def _check_store(gs, triples):
    S = gs.Store(triples)
    want_stats = storage.statistics(triples)
    got = {s["pred_id"]: s for s in S.pred_stats()}
    assert sorted(got) == sorted(want_stats)
    for p, w in want_stats.items():
        assert (got[p]["nnz"], got[p]["nr_s"], got[p]["nr_o"]) == (w["nnz"], w["nr_s"], w["nr_o"])
    for side, key in ((0, "s"), (1, "o")):
        ref = storage.csr_by(triples, key)
        for p, (rid, ptr, ent) in ref.items():
            g_rid, g_ptr, g_ent = S.export(p, side)
            assert np.array_equal(g_rid, rid), (p, side)
            assert np.array_equal(g_ptr, ptr), (p, side)
            assert np.array_equal(g_ent, ent), (p, side)
    info = S.info()
    assert info["n_unique"] == storage.unique_triples(triples).shape[0]
    assert info["n_input"] == np.asarray(triples).shape[0]
    return S


def test_dg_matrices(gs):
    g = golden("dg_example.json")
    S = _check_store(gs, np.array(g["cube_spo"], dtype=np.int32))
    for h, M in g["matrices"].items():
        rid, ptr, ent = S.export(int(h), 0)
        pairs = [[int(rid[r]), int(ent[j])] for r in range(len(rid)) for j in range(ptr[r], ptr[r + 1])]
        assert pairs == M


def test_tiny_graph_dense_rows(gs):
    t = synth.make_graph("tiny")
    S = _check_store(gs, t)
    assert S.info()["n_dense_rows_s"] > 0


def test_sparse_ids_use_row_search(gs):
    t = synth.make_graph("tiny").astype(np.int64)
    t[:, 0] *= 997
    t[:, 2] *= 991
    S = _check_store(gs, t.astype(np.int32))
    info = S.info()
    assert info["n_dense_rows_s"] == 0 and info["n_dense_rows_o"] == 0


def test_duplicates_removed(gs):
    rng = np.random.default_rng(0)
    t = synth.small_random_graph(50, 4, 400, seed=3)
    dup = np.concatenate([t, t[rng.integers(0, len(t), 300)]])
    rng.shuffle(dup)
    S = _check_store(gs, dup)
    assert S.info()["n_unique"] == len(t)


def test_wide_ids_two_pass_sort(gs):
    # slot bits + 2 * id bits > 64 exercises the two-pass sort
    rng = np.random.default_rng(1)
    n = 5000
    t = np.stack([rng.integers(0, 2**31 - 1, n), rng.integers(0, 9, n) * 1000003, rng.integers(0, 2**31 - 1, n)], 1)
    t[:100, 0] = 2**31 - 1
    _check_store(gs, t.astype(np.int32))


def test_single_predicate_and_self_loops(gs):
    t = np.array([(1, 42, 1), (1, 42, 2), (2, 42, 2), (3, 42, 1), (0, 42, 0)], dtype=np.int32)
    _check_store(gs, t)


def test_empty_and_invalid(gs):
    S = gs.Store(np.zeros((0, 3), np.int32))
    assert S.info()["n_unique"] == 0
    with pytest.raises(gs.GsmatError) as e:
        gs.Store(np.array([(1, 2, -3)], dtype=np.int32))
    assert e.value.code == 1


def test_device_input(gs):
    import torch

    t = synth.make_graph("tiny")
    S = gs.Store(torch.from_numpy(np.array(t, copy=True)).cuda())
    assert S.info()["n_unique"] == len(t)


def test_ragged_sizes(gs):
    for n in (1, 2, 3, 1023, 1024, 1025, 3071, 3072, 3073, 4097):
        t = synth.small_random_graph(200, 3, n, seed=n)
        _check_store(gs, t)


def test_many_distinct_predicates(gs):
    # more distinct predicates than the build's hash sets hold (sort path),
    # and a count that fits them (set path), with predicate ids spread wide
    rng = np.random.default_rng(11)
    for n_pred in (5000, 900):
        n = 20_000
        preds = rng.choice(2**30, size=n_pred, replace=False)
        t = np.stack([rng.integers(0, 3000, n), preds[rng.integers(0, n_pred, n)], rng.integers(0, 3000, n)], 1)
        S = _check_store(gs, t.astype(np.int32))
        assert S.info()["n_predicates"] == len(np.unique(t[:, 1]))
