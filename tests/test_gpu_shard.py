"""Row sharding of one query, shards run one after another on one GPU:
the shards partition the result exactly (GPU)."""

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


def _check(gs, S, pats, V, want, n_shards):
    full_plan = S.query(pats, V, flags=gs.PLAN_ORDER).to_numpy()
    parts = [S.query_shard(pats, k, n_shards, n_vars=V) for k in range(n_shards)]
    # sorted shards merge into the full sorted result (device merge)
    merged = gs.merge_tables(parts).to_numpy()
    assert merged.shape == want.shape and np.array_equal(merged, want)
    # plan-order shards follow each other: back to back they are the full table
    plan = [S.query_shard(pats, k, n_shards, n_vars=V, flags=gs.PLAN_ORDER).to_numpy() for k in range(n_shards)]
    cat = np.concatenate(plan, axis=0) if plan else full_plan
    assert np.array_equal(cat, full_plan)
    counts = [S.query_shard(pats, k, n_shards, n_vars=V, flags=gs.COUNT_ONLY).rows for k in range(n_shards)]
    assert sum(counts) == want.shape[0]
    # the first step's rows are split near-equally
    total = S.query(pats, V).stats()["rows"][0]
    if total >= 0:  # (-1: an absent predicate, nothing ran)
        first = [p.stats()["rows"][0] for p in parts]
        assert sum(first) == total and max(first) - min(first) <= 1


@pytest.mark.parametrize("n_shards", [1, 2, 3, 7])
def test_shards_tiny_workload(gs, tiny, n_shards):
    t, ix, S, qs = tiny
    for q in qs:
        _check(gs, S, q.patterns, q.n_vars, ix.query(q), n_shards)


@pytest.mark.parametrize("seed", range(8))
def test_shards_random_bgps(gs, tiny, seed):
    t, ix, S, qs = tiny
    rng = np.random.default_rng(3000 + seed)
    done = 0
    while done < 6:
        pats, V = random_bgp(rng, t, n_vars_max=4, n_pats_max=4, p_const=0.3)
        if V == 0:
            continue
        try:
            want = ix.query(pats, V, row_limit=2_000_000)
        except oracle.OracleError:
            continue
        _check(gs, S, pats, V, want, int(rng.integers(2, 6)))
        done += 1


def test_shard_arguments_and_merge_errors(gs, tiny):
    t, ix, S, qs = tiny
    q = qs[0]
    for k, n in ((0, 0), (2, 2), (-1, 2), (0, (1 << 20) + 1)):
        with pytest.raises(gs.GsmatError) as e:
            S.query_shard(q, k, n)
        assert e.value.code == 1
    a = S.query(qs[0])
    b = S.query(qs[1])
    if a.col_vars != b.col_vars:
        with pytest.raises(gs.GsmatError):
            gs.merge_tables([a, b])
    with pytest.raises(gs.GsmatError):
        gs.merge_tables([S.query(q, flags=gs.COUNT_ONLY)])
    # more shards than first-step rows: the extra shards are empty
    one = gs.Store(np.array([(1, 5, 2), (2, 5, 3)], dtype=np.int32))
    parts = [one.query_shard([(0, 5, 1, 1, 1)], k, 5, n_vars=2) for k in range(5)]
    # shard k keeps rows [2k/5, 2(k+1)/5) of the two: 0, 0, 1, 0, 1 rows
    assert [p.rows for p in parts] == [0, 0, 1, 0, 1]
    assert gs.merge_tables(parts).to_numpy().tolist() == [[1, 2], [2, 3]]


def _rank_worker(rank, world, port, q):
    """One rank: its shard of each tiny query on the device, copied to a host
    tensor and gathered to rank 0 over gloo (the ranks' kernels never wait
    on one another; only the host collectives do)."""
    import os
    import sys

    import torch
    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    import synth as sy
    import paper_1807_07691_b300 as g

    t = sy.make_graph("tiny")
    S = g.Store(t)
    ok = []
    for qq in sy.make_queries("tiny", t):
        part = S.query_shard(qq.patterns, rank, world, n_vars=qq.n_vars, flags=g.PLAN_ORDER).to_torch().cpu()
        got = g.gather_shards(part, dst=0)
        if rank == 0:
            whole = S.query(qq.patterns, qq.n_vars, flags=g.PLAN_ORDER).to_numpy()
            ok.append(bool(np.array_equal(got.numpy(), whole)))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ok))


def test_rank_shards_gathered_over_gloo(gs):
    import socket

    import torch.multiprocessing as mp

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] and all(res[0][1]) and res[1][1] == []
