"""The onesweep radix sort (qb_sort_pairs) against numpy's stable argsort:
bit-exact keys and values, stability under duplicates, ragged sizes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def run_sort(keys_np, vals_np, end_bit, digit_bits):
    import torch
    from paper_2605_04844_gb300 import _native as N
    n = len(keys_np)
    k = torch.from_numpy(keys_np.view(np.int64).copy()).cuda() if n else torch.zeros(1, dtype=torch.int64).cuda()
    v = torch.from_numpy(vals_np.view(np.int32).copy()).cuda() if n else torch.zeros(1, dtype=torch.int32).cuda()
    ka, va = torch.empty_like(k), torch.empty_like(v)
    sb = N.qb_sort_scratch_bytes(n, end_bit, digit_bits)
    scratch = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
    off = (-scratch.data_ptr()) % 256
    scratch = scratch[off:off + sb]
    alt = N.qb_sort_pairs(k, v, ka, va, n, end_bit, digit_bits, scratch)
    torch.cuda.synchronize()
    rk, rv = (ka, va) if alt else (k, v)
    return rk.cpu().numpy()[:n].view(np.uint64), rv.cpu().numpy()[:n].view(np.uint32)


def reference(keys, vals, end_bit):
    mask = np.uint64((1 << end_bit) - 1) if end_bit < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(keys & mask, kind="stable")
    return keys[order], vals[order]


@pytest.mark.parametrize("n", [0, 1, 7, 4095, 4096, 4097, 65_537, 1_000_003])
@pytest.mark.parametrize("digit_bits", [8, 11])
def test_sort_random(n, digit_bits):
    rng = np.random.default_rng(n + digit_bits)
    end_bit = 44
    keys = rng.integers(0, 1 << end_bit, n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    k, v = run_sort(keys, vals, end_bit, digit_bits)
    rk, rv = reference(keys, vals, end_bit)
    np.testing.assert_array_equal(k, rk)
    np.testing.assert_array_equal(v, rv)


@pytest.mark.parametrize("digit_bits", [8, 9, 10, 11])
@pytest.mark.parametrize("end_bit", [31, 39, 45, 51, 64])
def test_sort_duplicates_stable(digit_bits, end_bit):
    rng = np.random.default_rng(end_bit * 17 + digit_bits)
    n = 300_001
    # few distinct keys: long runs test stability and look-back across tiles
    base = rng.integers(0, 1 << min(end_bit, 62), 37, dtype=np.uint64)
    keys = base[rng.integers(0, 37, n)]
    if end_bit == 64:
        keys[::3] |= np.uint64(1) << np.uint64(63)
    vals = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    k, v = run_sort(keys, vals, end_bit, digit_bits)
    rk, rv = reference(keys, vals, end_bit)
    np.testing.assert_array_equal(k, rk)
    np.testing.assert_array_equal(v, rv)


def test_sort_all_equal_and_presorted():
    n = 123_457
    keys = np.full(n, 12345, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint32)[::-1].copy()
    k, v = run_sort(keys, vals, 40, 8)
    np.testing.assert_array_equal(v, vals)
    keys = np.arange(n, dtype=np.uint64) * np.uint64(977)
    k, v = run_sort(keys, np.arange(n, dtype=np.uint32), 40, 11)
    np.testing.assert_array_equal(k, keys)
