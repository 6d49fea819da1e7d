"""Radix sort and scan primitives through the C ABI against numpy (GPU)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    torch.cuda.init()
    import paper_1807_07691_b300 as g

    return g, torch


@pytest.mark.parametrize("n", [0, 1, 2, 100, 3071, 3072, 3073, 100_000, 1_234_567])
@pytest.mark.parametrize("bits", [(0, 64), (0, 20), (8, 40)])
def test_radix_sort_pairs_stable(env, n, bits):
    g, torch = env
    rng = np.random.default_rng(n + bits[1])
    keys = rng.integers(0, 2**63, size=n, dtype=np.int64).view(np.uint64)
    if n > 10:
        keys[: n // 3] = keys[0]  # many equal keys: stability matters
    vals = np.arange(n, dtype=np.uint32)
    dk = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    g.radix_sort_u64(dk, dv, bits[0], bits[1])
    torch.cuda.synchronize()
    b0, b1 = bits
    mask = np.uint64((1 << (b1 - b0)) - 1) if b1 - b0 < 64 else np.uint64(2**64 - 1)
    digit = (keys >> np.uint64(b0)) & mask
    order = np.argsort(digit, kind="stable")
    assert np.array_equal(dk.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(dv.cpu().numpy().view(np.uint32), vals[order])


def test_radix_sort_keys_only(env):
    g, torch = env
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 2**40, size=500_001, dtype=np.int64)
    dk = torch.from_numpy(keys.copy()).cuda()
    g.radix_sort_u64(dk, None, 0, 40)
    assert np.array_equal(dk.cpu().numpy(), np.sort(keys))


@pytest.mark.parametrize("n", [0, 1, 5, 2047, 2048, 2049, 1_000_003])
def test_exclusive_scan(env, n):
    g, torch = env
    rng = np.random.default_rng(n)
    x = rng.integers(0, 1000, size=n).astype(np.int32)
    dx = torch.from_numpy(x).cuda()
    out = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    g.exclusive_scan_i32(dx, out)
    want = np.concatenate([[0], np.cumsum(x, dtype=np.int64)])
    assert np.array_equal(out.cpu().numpy(), want)


def test_scan_total_beyond_int32(env):
    g, torch = env
    n = 3_000_000
    x = np.full(n, 2**30, dtype=np.int32)
    x[::7] = 5
    out = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    g.exclusive_scan_i32(torch.from_numpy(x).cuda(), out)
    want = np.concatenate([[0], np.cumsum(x, dtype=np.int64)])
    assert np.array_equal(out.cpu().numpy(), want)
    assert want[-1] > 2**31


# (V, m, bits, n, value range): single chunk with gathered columns; two and
# three chunks; a one-pass chunk that is not the last one sorted (SrcRows ->
# permutation) and a one-pass final chunk; tile edges; narrow value ranges
# so that equal keys are common and stability decides the order; both sides
# of the one-CTA size limit (2048 rows, keys of up to two words); gathered
# columns as one- and two-word records, as separate columns (more than
# eight), and read in place when the permutation keeps runs (all keys equal);
# non-key columns that fit 64 bits carried through the passes as a payload.
SORT_ROWS_CASES = [
    (3, 1, 20, 100_000, 1 << 20),
    (5, 4, 20, 300_001, 1 << 20),
    (5, 4, 20, 300_001, 3),
    (4, 4, 3, 50_000, 8),
    (1, 1, 5, 10_000, 32),
    (2, 1, 5, 3073, 32),
    (6, 6, 31, 70_000, 1 << 31),
    (24, 23, 3, 20_000, 8),
    (3, 2, 17, 0, 1),
    (3, 2, 17, 1, 1 << 17),
    (3, 2, 17, 2, 1 << 17),
    (2, 2, 12, 3071, 1 << 12),
    (2, 2, 12, 3072, 1 << 12),
    (6, 6, 31, 5000, 1 << 31),
    (10, 2, 20, 50_000, 1 << 20),
    (12, 1, 20, 40_000, 1 << 20),
    (7, 3, 20, 2048, 50),
    (7, 3, 20, 2049, 50),
    (6, 5, 20, 1500, 1 << 20),
    (6, 6, 20, 2000, 4),
    (5, 1, 20, 100_000, 1),
    (5, 2, 20, 300_001, 1 << 20),
    (5, 3, 20, 100_000, 7),
    (4, 1, 21, 70_000, 1 << 21),
    (3, 2, 31, 10_000, 1 << 31),
]


@pytest.mark.parametrize("flags", [0, 1, 2])  # by size, carried, gathered
@pytest.mark.parametrize("V,m,bits,n,hi", SORT_ROWS_CASES)
def test_sort_rows_matches_stable_lexsort(env, V, m, bits, n, hi, flags):
    g, torch = env
    rng = np.random.default_rng(V * 1000 + m * 100 + bits + n)
    cols = [rng.integers(0, hi, size=n, dtype=np.int64).astype(np.int32) for _ in range(V)]
    d = [torch.from_numpy(c.copy()).cuda() for c in cols]
    out = g.sort_rows(d, m, bits, flags=flags)
    torch.cuda.synchronize()
    # np.lexsort is stable and takes its primary key last
    order = np.lexsort(cols[m - 1::-1]) if n else np.zeros(0, np.int64)
    for v in range(V):
        assert np.array_equal(out[v].cpu().numpy(), cols[v][order]), v


def test_sort_rows_rejects_bad_arguments(env):
    g, torch = env
    c = [torch.zeros(4, dtype=torch.int32, device="cuda") for _ in range(2)]
    for m, bits, flags in ((3, 8, 0), (0, 8, 0), (1, 0, 0), (1, 32, 0), (1, 8, 3)):
        with pytest.raises(g.GsmatError) as e:
            g.sort_rows(c, m, bits, flags=flags)
        assert e.value.code == 1


def test_launch_count_counts_kernels(env):
    g, torch = env
    keys = torch.randint(0, 2**40, (100_000,), device="cuda", dtype=torch.int64)
    c0 = g.launch_count()
    g.radix_sort_u64(keys, None, 0, 40)
    torch.cuda.synchronize()
    assert g.launch_count() - c0 == 1 + 5  # digit histogram + five 8-bit passes


# Sorts of at least 2^23 keys with a payload run the large-sort pass shape
# (larger tiles, atomicOr ranking); both sides of the threshold, and the
# row reorder's carried (64-bit payload) and gathered (row-index payload)
# paths above it.
@pytest.mark.parametrize("n", [(1 << 23) - 1, (1 << 23) + 12_345])
def test_radix_sort_pairs_large_shape(env, n):
    g, torch = env
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 1 << 40, size=n, dtype=np.int64)
    keys[: n // 4] = keys[7]  # a long run of equal keys: stability
    vals = np.arange(n, dtype=np.uint32)
    dk = torch.from_numpy(keys.copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    g.radix_sort_u64(dk, dv, 0, 40)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(dk.cpu().numpy(), keys[order])
    assert np.array_equal(dv.cpu().numpy().view(np.uint32), vals[order])


@pytest.mark.parametrize("flags", [1, 2])  # carried, gathered
def test_sort_rows_large_shape(env, flags):
    g, torch = env
    n, V, m, bits = 9_000_001, 4, 2, 21  # 42 key bits + a 24-bit row index exceed one word
    rng = np.random.default_rng(77 + flags)
    cols = [rng.integers(0, 1 << bits, size=n, dtype=np.int64).astype(np.int32) for _ in range(V)]
    cols[0][: n // 3] = 5  # equal leading keys
    d = [torch.from_numpy(c.copy()).cuda() for c in cols]
    out = g.sort_rows(d, m, bits, flags=flags)
    order = np.lexsort(cols[m - 1::-1])
    for v in range(V):
        assert np.array_equal(out[v].cpu().numpy(), cols[v][order]), v
