"""Served evaluation (continuous batching): each result is the same alone
and in the mix (GPU)."""

import threading

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
    S = gs.Store(t)
    items = [(q.patterns, q.n_vars) for q in synth.make_queries("tiny", t)]
    rng = np.random.default_rng(31)
    ix = oracle.OracleIndex(t)
    while len(items) < 200:
        pats, V = random_bgp(rng, t, n_vars_max=4, n_pats_max=4, p_const=0.5)
        try:
            ix.query(pats, V, row_limit=500_000)  # keep the mix small enough
        except oracle.OracleError:
            continue
        items.append((pats, V))
    alone = [S.query(p, v).to_numpy() for p, v in items]
    return S, items, alone


def _run(srv, items):
    tickets = [srv.submit(p, v) for p, v in items]
    for t in tickets:
        assert srv.wait(t)
    return tickets


def test_results_same_alone_and_in_the_mix(gs, tiny):
    S, items, alone = tiny
    srv = gs.Server(S, max_batch=32, slots=4, batch_lone=True)
    tickets = _run(srv, items)
    for t, want in zip(tickets, alone):
        got = srv.to_numpy(t)
        assert got.shape == want.shape and np.array_equal(got, want)
        rows, cols, lat = srv.result(t)
        assert lat > 0
        srv.release(t)
    st = srv.stats()
    assert st["completed"] == len(items) and st["failed"] == 0 and st["batches"] >= len(items) // 32
    srv.close()


def test_cost_plan_server(gs, tiny):
    # micro-batches, the lone lane and the admission estimate all plan by cost
    S, items, alone = tiny
    srv = gs.Server(S, max_batch=16, slots=2, batch={"plan_cost": 1})
    tickets = _run(srv, items)
    for t, want in zip(tickets, alone):
        assert np.array_equal(srv.to_numpy(t), want)
        srv.release(t)
    assert srv.stats()["failed"] == 0
    srv.close()
    with pytest.raises(gs.GsmatError):
        gs.Server(S, batch={"plan_cost": 3})


def test_tight_budget_and_concurrent_submitters(gs, tiny):
    S, items, alone = tiny
    srv = gs.Server(S, max_batch=8, slots=2, budget_bytes=1 << 20)
    out = {}

    def worker(lo, hi):
        for i in range(lo, hi):
            out[i] = srv.submit(*items[i])

    ths = [threading.Thread(target=worker, args=(k * 50, (k + 1) * 50)) for k in range(len(items) // 50)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    for i, t in out.items():
        assert srv.wait(t)
        assert np.array_equal(srv.to_numpy(t), alone[i])
    assert srv.stats()["in_flight_bytes"] == 0
    srv.close()


def test_close_with_pending_work(gs, tiny):
    S, items, alone = tiny
    srv = gs.Server(S, max_batch=4, slots=1)
    for p, v in items:
        srv.submit(p, v)
    srv.close()  # finishes what is in flight, fails the rest, does not hang


def test_sparse_requests_take_a_direct_lane(gs, tiny):
    # sparse arrivals (2 ms apart), each finding the queue empty: each runs
    # as gsmat_query on a direct lane's stream, with the same result
    import time

    S, items, alone = tiny
    srv = gs.Server(S)
    for (p, v), want in list(zip(items, alone))[:20]:
        time.sleep(0.002)
        t = srv.submit(p, v)
        assert srv.wait(t)
        got = srv.to_numpy(t)
        assert got.shape == want.shape and np.array_equal(got, want)
        rows, cols, lat = srv.result(t)
        assert rows == want.shape[0] and lat > 0
        srv.release(t)
    st = srv.stats()
    assert st["direct"] == 20 and st["batches"] == 0 and st["completed"] == 20
    srv.close()


def test_burst_splits_between_lanes_and_micro_batches(gs, tiny):
    """A burst: the first requests find idle lanes, the ones queued behind
    them form micro-batches; every result is the one alone."""
    import time

    S, items, alone = tiny
    srv = gs.Server(S, max_batch=16, slots=2, lanes=3)
    tickets = []
    for p, v in items[:3]:  # spaced out: each finds the queue empty
        time.sleep(0.003)
        tickets.append(srv.submit(p, v))
    tickets += [srv.submit(p, v) for p, v in items[3:]]  # back to back: they queue up
    for t in tickets:
        assert srv.wait(t)
    for t, want in zip(tickets, alone):
        assert np.array_equal(srv.to_numpy(t), want)
        srv.release(t)
    st = srv.stats()
    assert st["completed"] == len(items) and st["failed"] == 0
    assert st["direct"] >= 1 and st["batches"] >= 1
    srv.close()
    with pytest.raises(gs.GsmatError):
        gs.Server(S, lanes=65)
