"""The C ABI library loads, exports every declared symbol, and its host
planner agrees with the oracle's restatement of Alg. 1 (CPU only)."""

import ctypes

import numpy as np
import pytest

import oracle.planner as oplan
import synth
from oracle import storage
from tests.helpers import golden


@pytest.fixture(scope="module")
def gs():
    import paper_1807_07691_b300 as g

    return g


def test_library_exports_every_header_symbol(gs):
    names = gs.header_functions()
    assert len(names) >= 20
    lib = gs.lib()
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_strerror_and_version(gs):
    lib = gs.lib()
    assert lib.gsmat_version() >= 100
    for code in range(7):
        assert lib.gsmat_strerror(code)
    assert lib.gsmat_strerror(99) == b"unknown status"


def test_plan_rejects_bad_bgps(gs):
    with pytest.raises(gs.GsmatError) as e:
        gs.plan([(0, 5, 1, 1, 1)], [1], [dict(nnz=1, nr_s=1, nr_o=1)], n_vars=3)
    assert e.value.code == 1
    with pytest.raises(gs.GsmatError) as e:
        gs.plan(np.array([[0, 5, 1, 1, 1, 1]]), [1], [dict(nnz=1, nr_s=1, nr_o=1)], n_vars=2)
    assert e.value.code == 2


def test_plan_matches_paper_bgp_sequence(gs):
    g = golden("dg_example.json")
    st = storage.statistics(np.array(g["cube_spo"]))
    stats = [st[p[1]] for p in g["query"]]
    keys = [s["nnz"] for s in stats]
    order, kinds, est = gs.plan(g["query"], keys, stats, n_vars=4)
    assert order == g["plan_order"]
    o_order = oplan.plan_order(g["query"], keys)
    o_est, _, o_kinds = oplan.estimate(g["query"], o_order, keys, stats)
    assert kinds == o_kinds
    assert np.allclose(est, o_est, rtol=1e-12)


def _random_case(rng):
    n = int(rng.integers(1, 9))
    nv = int(rng.integers(1, 6))
    pats = []
    for _ in range(n):
        ends = []
        for _e in range(2):
            if rng.random() < 0.2:
                ends.append((int(rng.integers(0, 100)), 0))
            else:
                ends.append((int(rng.integers(nv)), 1))
        pats.append((ends[0][0], int(rng.integers(0, 4)), ends[1][0], ends[0][1], ends[1][1]))
    used = sorted({p[0] for p in pats if p[3]} | {p[2] for p in pats if p[4]})
    remap = {v: i for i, v in enumerate(used)}
    pats = [(remap[s] if sv else s, p, remap[o] if ov else o, sv, ov) for (s, p, o, sv, ov) in pats]
    keys = rng.integers(0, 50, size=n).tolist()
    stats = [dict(nnz=int(rng.integers(0, 1000)), nr_s=int(rng.integers(0, 50)), nr_o=int(rng.integers(0, 50)))
             for _ in range(n)]
    return pats, len(used), keys, stats


@pytest.mark.parametrize("seed", range(25))
def test_plan_matches_oracle_planner(gs, seed):
    rng = np.random.default_rng(seed)
    pats, nv, keys, stats = _random_case(rng)
    order, kinds, est = gs.plan(pats, keys, stats, n_vars=nv)
    o_order = oplan.plan_order(pats, keys)
    assert order == o_order
    o_est, _, o_kinds = oplan.estimate(pats, o_order, keys, stats)
    assert kinds == o_kinds
    assert np.allclose(est, o_est, rtol=1e-12, atol=0)


@pytest.mark.parametrize("seed", range(40))
def test_cost_plan_matches_oracle(gs, seed):
    """gsmat_plan_cost = the oracle's least-cost connected order, bit for bit
    (the argmin is taken in fp64 on both sides, step-order sums)."""
    rng = np.random.default_rng(1000 + seed)
    pats, nv, keys, stats = _random_case(rng)
    order, kinds, est = gs.plan(pats, keys, stats, n_vars=nv, cost=True)
    o_order = oplan.cost_plan_order(pats, keys, stats)
    assert order == o_order
    o_est, _, o_kinds = oplan.estimate(pats, o_order, keys, stats)
    assert kinds == o_kinds
    assert est == o_est


def test_cost_plan_worked_chain_and_limits(gs):
    # the chain A-B-C of the oracle's worked example: Alg. 1 costs 30100,
    # the least-cost connected order (B, C, A) 15300
    pats = [(0, 1, 1, 1, 1), (1, 2, 2, 1, 1), (2, 3, 3, 1, 1)]
    stats = [dict(nnz=100, nr_s=100, nr_o=1), dict(nnz=150, nr_s=1, nr_o=150), dict(nnz=200, nr_s=200, nr_o=200)]
    keys = [100, 150, 200]
    assert gs.plan(pats, keys, stats, n_vars=4)[0] == [0, 1, 2]
    order, kinds, est = gs.plan(pats, keys, stats, n_vars=4, cost=True)
    assert order == [1, 2, 0] and est == [150.0, 150.0, 15000.0]
    # above GSMAT_PLAN_COST_MAX patterns: Alg. 1
    n = gs.PLAN_COST_MAX + 1
    chain = [(i, 1, i + 1, 1, 1) for i in range(n)]
    k = list(range(n, 0, -1))
    st = [dict(nnz=10, nr_s=5, nr_o=5)] * n
    assert gs.plan(chain, k, st, n_vars=n + 1, cost=True) == gs.plan(chain, k, st, n_vars=n + 1)
    with pytest.raises(gs.GsmatError) as e:
        gs.plan([(0, 5, 1, 1, 1)], [1], [dict(nnz=1, nr_s=1, nr_o=1)], n_vars=3, cost=True)
    assert e.value.code == 1


def test_cost_plan_on_tiny_workload(gs):
    t = synth.make_graph("tiny")
    st = storage.statistics(t)
    for q in synth.make_queries("tiny", t):
        stats = [st[p[1]] for p in q.patterns]
        keys = [s["nnz"] for s in stats]
        order, kinds, est = gs.plan(q, keys, stats, cost=True)
        assert order == oplan.cost_plan_order(q.patterns, keys, stats)


def test_plan_on_tiny_workload(gs):
    t = synth.make_graph("tiny")
    st = storage.statistics(t)
    for q in synth.make_queries("tiny", t):
        stats = [st[p[1]] for p in q.patterns]
        keys = [s["nnz"] for s in stats]
        order, kinds, est = gs.plan(q, keys, stats)
        assert order == oplan.plan_order(q.patterns, keys)


def test_lazy_package_names_resolve(gs):
    import paper_1807_07691_b300 as pkg

    for name in dir(pkg):
        if name not in ("build", "gsmat"):
            assert getattr(pkg, name) is getattr(gs, name), name


def test_primitives_refuse_host_and_mismatched_tensors(gs):
    """The device primitives' bindings refuse what the library would
    dereference wrongly on the device: host tensors, wrong dtypes, short or
    strided buffers (checked before any library call, so CPU only)."""
    import torch

    k64 = torch.zeros(8, dtype=torch.int64)
    i32 = torch.zeros(8, dtype=torch.int32)
    for call in (lambda: gs.radix_sort_u64(k64),
                 lambda: gs.exclusive_scan_i32(i32, torch.zeros(9, dtype=torch.int64)),
                 lambda: gs.exclusive_scan_i32_noalloc(i32, torch.zeros(9, dtype=torch.int64)),
                 lambda: gs.sort_rows([i32, i32], 1, 8),
                 lambda: gs.sort_rows([torch.zeros(8, dtype=torch.float32)], 1, 8)):
        with pytest.raises(ValueError):
            call()
    from paper_1807_07691_b300 import gsmat

    with pytest.raises(ValueError):
        gsmat._require(k64, (torch.int64,), 0, "keys")  # host tensor
    with pytest.raises(ValueError):
        gsmat._require(k64[::2], (torch.int64,), 0, "keys")


def test_wait_expiry_selftest_rejects_bad_poll_limits(gs):
    """Argument checks of the bounded-wait self-test happen on the host,
    before any device work."""
    lib = gs.lib()
    for bad in (0, -1, (1 << 22) + 1):
        assert lib.gsmat_selftest_wait_expiry(bad, None) == 1  # GSMAT_ERR_INVALID_ARG
        assert b"poll limit" in lib.gsmat_last_error()


def test_tile_setters_check_their_arguments_on_the_host(gs):
    lib = gs.lib()
    assert lib.gsmat_store_set_tiles(None, None) == 1
    assert lib.gsmat_store_get_tiles(None, None) == 1
    assert lib.gsmat_store_tune(None, None, 0, None, None) == 1
