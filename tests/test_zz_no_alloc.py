"""The exclusive scan that allocates nothing, checked against the regular one
through the C ABI (GPU).

gsmat_exclusive_scan_i32_noalloc exists for callers that cannot allocate
device memory: code running under a fixed device-memory budget that another
allocator already owns, or on a latency-critical path that must not enter
the driver's allocator.  It keeps its scratch in a static device array that
every call reuses, so each call must clear what it uses; two calls in a row
with different sizes and data must both match gsmat_exclusive_scan_i32
exactly (integer sums: tolerance zero).

This file is collected last so that a run stopping at the first failure has
run everything else; it also passes alone in a fresh process.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    torch.cuda.init()
    import paper_1807_07691_b300 as gs

    return gs, torch


def _scan_both(gs, torch, x, stream=None):
    lib = gs.lib()
    stream = stream or torch.cuda.current_stream()
    st = ctypes.c_void_p(stream.cuda_stream)
    n = x.numel()
    ref = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
    out = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
    assert lib.gsmat_exclusive_scan_i32(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(ref.data_ptr()), n, st) == 0
    assert lib.gsmat_exclusive_scan_i32_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), n,
                                                st) == 0
    stream.synchronize()
    return ref.cpu().numpy(), out.cpu().numpy()


def test_noalloc_scan_matches_regular_scan_on_consecutive_calls(env):
    gs, torch = env
    rng = np.random.default_rng(5)
    for n in (5_000_003, 3_000_001, 2049):  # shrinking: stale descriptors would show
        x = torch.from_numpy(rng.integers(0, 1 << 20, size=n).astype(np.int32)).cuda()
        ref, out = _scan_both(gs, torch, x)
        assert np.array_equal(ref, out), n
        assert out[-1] == int(x.sum().item())


def test_noalloc_scan_of_nothing_writes_a_zero_total(env):
    gs, torch = env
    x = torch.zeros(0, dtype=torch.int32, device="cuda")
    ref, out = _scan_both(gs, torch, x)
    assert ref.tolist() == out.tolist() == [0]


def test_noalloc_scan_on_a_side_stream(env):
    """Work ordered on a stream other than the current one: the clearing
    memsets and the kernel follow that stream's order."""
    gs, torch = env
    rng = np.random.default_rng(6)
    side = torch.cuda.Stream()
    for n in (1_000_003, 40_000):
        x = torch.from_numpy(rng.integers(0, 1 << 16, size=n).astype(np.int32)).cuda()
        side.wait_stream(torch.cuda.current_stream())
        ref, out = _scan_both(gs, torch, x, stream=side)
        assert np.array_equal(ref, out), n


def test_noalloc_scan_at_its_maximum_size(env):
    gs, torch = env
    n = gs.exclusive_scan_i32_noalloc_max()
    x = torch.randint(0, 3, (n,), dtype=torch.int32, device="cuda")
    ref, out = _scan_both(gs, torch, x)
    assert np.array_equal(ref, out)


def test_noalloc_scan_rejects_sizes_beyond_its_maximum(env):
    gs, torch = env
    lib = gs.lib()
    x = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    too_big = gs.exclusive_scan_i32_noalloc_max() + 1
    # rejected on the host before any device work
    rc = lib.gsmat_exclusive_scan_i32_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                              too_big, ctypes.c_void_p(0))
    assert rc == 4  # GSMAT_ERR_CAPACITY
    assert b"maximum" in lib.gsmat_last_error()
