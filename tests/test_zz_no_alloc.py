"""qb_sort_pairs_noalloc: the pair sort for callers that may not allocate
device memory (for example a plug-in whose host application owns all device
memory, or a render loop that must not stall on cudaMalloc).  Its scratch is
a fixed array inside the library, so it must give exactly the results of the
allocating qb_sort_pairs, call after call, even though the array keeps the
previous call's contents.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _sort_allocating(k, v, n, end_bit, digit_bits):
    import torch
    from paper_2605_04844_gb300 import _native as N
    ka, va = torch.empty_like(k), torch.empty_like(v)
    kk, vv = k.clone(), v.clone()
    sb = N.qb_sort_scratch_bytes(n, end_bit, digit_bits)
    raw = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
    off = (-raw.data_ptr()) % 256
    alt = N.qb_sort_pairs(kk, vv, ka, va, n, end_bit, digit_bits, raw[off:off + sb])
    return (ka, va) if alt else (kk, vv)


def _sort_noalloc(k, v, n, end_bit, digit_bits):
    import torch
    from paper_2605_04844_gb300 import _native as N
    ka, va = torch.empty_like(k), torch.empty_like(v)
    kk, vv = k.clone(), v.clone()
    alt = N.qb_sort_pairs_noalloc(kk, vv, ka, va, n, end_bit, digit_bits)
    return (ka, va) if alt else (kk, vv)


@pytest.mark.parametrize("digit_bits", [8, 11])
def test_noalloc_sort_matches_allocating_sort_on_consecutive_calls(digit_bits):
    import torch
    end_bit = 44
    # two calls in a row, the second smaller, so stale scratch from the first
    # call would show up if anything were not cleared
    for call, n in enumerate((1_000_003, 250_001)):
        rng = np.random.default_rng(100 + call + digit_bits)
        keys = rng.integers(0, 1 << end_bit, n, dtype=np.uint64)
        keys[1::2] = keys[0::2][: len(keys[1::2])]  # duplicate keys test stability
        vals = np.arange(n, dtype=np.uint32)
        k = torch.from_numpy(keys.view(np.int64).copy()).cuda()
        v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
        ka, va = _sort_allocating(k, v, n, end_bit, digit_bits)
        kb, vb = _sort_noalloc(k, v, n, end_bit, digit_bits)
        torch.cuda.synchronize()
        # integer work: bit-exact
        assert torch.equal(ka[:n], kb[:n]), f"keys differ on call {call}"
        assert torch.equal(va[:n], vb[:n]), f"values differ on call {call}"
        order = np.argsort(keys, kind="stable")
        np.testing.assert_array_equal(kb[:n].cpu().numpy().view(np.uint64), keys[order])


def test_noalloc_sort_rejects_sizes_beyond_the_static_array():
    import torch
    from paper_2605_04844_gb300 import _native as N
    cap = N.load().qb_sort_pairs_noalloc_max_scratch()
    assert cap == 16 << 20
    n = 20_000_000  # needs more scratch than the array holds at 44 bits / 8-bit digits
    assert N.qb_sort_scratch_bytes(n, 44, 8) - 256 > cap
    k = torch.zeros(1, dtype=torch.int64, device="cuda")
    v = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(N.QbError) as ei:
        N.qb_sort_pairs_noalloc(k, v, k, v, n, 44, 8)
    assert ei.value.status == N.QB_ERR_INVALID_ARG
    assert "static scratch" in str(ei.value)
