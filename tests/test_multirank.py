"""The benchmark's multi-rank path (replicas, max-over-ranks timing) with
world_size 2 on the gloo backend (CPU only)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys

    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank 1 is the slow one; rows add up
    ms, rows = bench.reduce_over_ranks(100.0 + 50.0 * rank, 1000 + rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, rows, bench.job_value(world, 3, 40, ms)))


def test_two_rank_reduction_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rows, value in res:
        assert ms == 150.0  # the slowest rank's time
        assert rows == 2001
        assert value == pytest.approx(2 * 3 * 40 / 0.150)


def test_single_process_is_identity():
    import bench

    assert bench.reduce_over_ranks(12.5, 7) == (12.5, 7)
    assert bench.job_value(1, 5, 40, 100.0) == pytest.approx(2000.0)


def _shard_worker(rank, world, port, q):
    import sys

    import numpy as np
    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    from paper_1807_07691_b300 import gsmat

    t = synth.make_graph("tiny")
    qq = synth.make_queries("tiny", t)[1]
    full = oracle.OracleIndex(t).query(qq)
    # rank r holds shard r: the r-th contiguous part, split as the library
    # splits the first relation (lo = rows * r // world)
    lo, hi = full.shape[0] * rank // world, full.shape[0] * (rank + 1) // world
    got = gsmat.gather_rows(full[lo:hi], dst=0)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, None if got is None else bool(np.array_equal(got, full)), full.shape[0]))


def test_two_rank_row_shards_gather_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] is True and res[1][1] is None and res[0][2] > 0


def _tensor_shard_worker(rank, world, port, q):
    import sys

    import numpy as np
    import torch
    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    from paper_1807_07691_b300 import gsmat

    t = synth.make_graph("tiny")
    full = oracle.OracleIndex(t).query(synth.make_queries("tiny", t)[1])
    out = []
    # near-equal shards as the library splits them, then uneven ones with an
    # empty shard, gathered once on rank 0 and once on the last rank
    for cuts, dst in (([full.shape[0] * r // world for r in range(world + 1)], 0),
                      ([0, 0] + [full.shape[0]] * (world - 1), world - 1)):
        part = torch.from_numpy(np.ascontiguousarray(full[cuts[rank]:cuts[rank + 1]]))
        got = gsmat.gather_shards(part, dst=dst)
        out.append(None if got is None else bool(np.array_equal(got.numpy(), full)))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out, full.shape[0]))


def test_two_rank_tensor_shard_gather_gloo():
    """gsmat.gather_shards: shard sizes exchanged, padded shards all-gathered
    as tensors (gloo here; NCCL with device tensors on GPUs)."""
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_tensor_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == [True, None] and res[1][1] == [None, True] and res[0][2] > 0
