"""Failure handling in the forms that fault no GPU (GPU).

* A bounded device wait that runs out: the library's scan kernel is run
  with one tile that never publishes its prefix (a flag nothing sets); its
  look-back waits give up after a short poll limit and the call returns
  GSMAT_ERR_DEVICE_CHECK, after which the same stream still computes
  correct results.
* Device allocation failure: an allocator hook that returns NULL at its
  k-th call, for every k of one store build and of one query.  Each such
  call returns GSMAT_ERR_OOM, frees everything it had allocated (the hook's
  live-allocation count returns to what it was), and the next call with a
  working hook gives the oracle's result.
"""

import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

OOM, DEVICE_CHECK = 3, 6


@pytest.fixture(scope="module")
def env():
    import torch

    torch.cuda.init()
    import paper_1807_07691_b300 as gs

    return gs, torch


def test_expired_wait_is_reported_and_the_stream_stays_usable(env):
    gs, torch = env
    lib = gs.lib()
    st = torch.cuda.current_stream()
    for limit in (1, 64, 4096):
        rc = lib.gsmat_selftest_wait_expiry(limit, ctypes.c_void_p(st.cuda_stream))
        assert rc == DEVICE_CHECK, (limit, rc, lib.gsmat_last_error())
        assert b"bounded wait" in lib.gsmat_last_error()
    # the context and the stream still work: a scan and a query right after
    x = torch.randint(0, 100, (1_000_003,), dtype=torch.int32, device="cuda")
    out = torch.empty(x.numel() + 1, dtype=torch.int64, device="cuda")
    gs.exclusive_scan_i32(x, out)
    torch.cuda.synchronize()
    want = np.concatenate([[0], np.cumsum(x.cpu().numpy().astype(np.int64))])
    assert np.array_equal(out.cpu().numpy(), want)
    t = synth.make_graph("tiny")
    q = synth.make_queries("tiny", t)[0]
    S = gs.Store(torch.from_numpy(np.array(t, copy=True)).cuda())
    assert np.array_equal(S.query(q).to_numpy(), oracle.OracleIndex(t).query(q))
    S.free()


class _FailingHook:
    """Allocator hook over torch's caching allocator that fails its
    `fail_at`-th call (counting from 0; None = never) and tracks live
    allocations."""

    def __init__(self, gs, torch):
        self.torch = torch
        self.calls = 0
        self.fail_at = None
        self.live = {}
        ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
        FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
        self._a = ALLOC(self._alloc)
        self._f = FREE(self._free)
        rc = gs.lib().gsmat_set_allocator(ctypes.cast(self._a, ctypes.c_void_p), ctypes.cast(self._f, ctypes.c_void_p),
                                          None)
        assert rc == 0

    def _alloc(self, nbytes, ctx, stream):
        k = self.calls
        self.calls += 1
        if self.fail_at is not None and k == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(max(nbytes, 1)), stream=int(stream or 0))
        self.live[int(p)] = int(nbytes)
        return p

    def _free(self, ptr, ctx, stream):
        self.live.pop(int(ptr))
        self.torch.cuda.caching_allocator_delete(int(ptr))


def test_allocation_failure_at_every_call_returns_oom_without_leaks(env):
    gs, torch = env
    t = synth.make_graph("tiny")
    qs = synth.make_queries("tiny", t)
    ix = oracle.OracleIndex(t)
    d_t = torch.from_numpy(np.array(t, copy=True)).cuda()
    hook = _FailingHook(gs, torch)
    try:
        # store build: count its allocations, then fail each one in turn
        c0 = hook.calls
        S = gs.Store(d_t)
        n_load = hook.calls - c0
        S.free()
        torch.cuda.synchronize()
        assert n_load > 0 and not hook.live
        for k in range(n_load):
            hook.fail_at = hook.calls + k
            with pytest.raises(gs.GsmatError) as e:
                gs.Store(d_t)
            assert e.value.code == OOM, (k, e.value)
            torch.cuda.synchronize()
            assert not hook.live, (k, len(hook.live))
        hook.fail_at = None
        S = gs.Store(d_t)
        held = len(hook.live)
        for q in (qs[0], qs[-1]):  # a chain and the triangle (intersect-expand)
            want = ix.query(q)
            c0 = hook.calls
            T = S.query(q)
            n_q = hook.calls - c0
            T.free()
            torch.cuda.synchronize()
            assert n_q > 0 and len(hook.live) == held
            for k in range(n_q):
                hook.fail_at = hook.calls + k
                with pytest.raises(gs.GsmatError) as e:
                    S.query(q)
                assert e.value.code == OOM, (q.name, k, e.value)
                torch.cuda.synchronize()
                assert len(hook.live) == held, (q.name, k)
            hook.fail_at = None
            T = S.query(q)
            assert np.array_equal(T.to_numpy(), want), q.name
            T.free()
        S.free()
        torch.cuda.synchronize()
        assert not hook.live
    finally:
        gs.lib().gsmat_set_allocator(None, None, None)
