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
