"""stiv_sort_pairs_static (the allocation-free sort) against stiv_sort_pairs.

Two calls in a row on different inputs: the second must not see the first
call's leftovers in the shared static scratch array.  The file name keeps it
last in collection; it also passes when run alone in a fresh process, where
its first call does the per-device set-up."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _sort_reference(S, keys, vals, bits):
    n = keys.numel()
    nb = S.stiv_sort_scratch_bytes(n)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    S.stiv_sort_pairs(torch.cuda.current_stream().cuda_stream, n, bits, keys.data_ptr(), vals.data_ptr(),
                      ko.data_ptr(), vo.data_ptr(), scratch.data_ptr(), nb)
    return ko, vo


def _sort_static(S, keys, vals, bits):
    n = keys.numel()
    ko = torch.full_like(keys, -1)
    vo = torch.full_like(vals, -1)
    S.stiv_sort_pairs_static(torch.cuda.current_stream().cuda_stream, n, bits, keys.data_ptr(), vals.data_ptr(),
                             ko.data_ptr(), vo.data_ptr())
    return ko, vo


def test_static_sort_matches_scratch_sort_twice():
    from paper_1812_04719_gb300 import stiv as S
    rng = np.random.default_rng(20181212)
    # first call larger than the second, so stale tiles of the first would show
    for n, bits in ((300_001, 53), (70_007, 30)):
        k = rng.integers(0, 1 << min(bits, 62), size=n, dtype=np.int64)
        k[rng.integers(0, n, size=n // 8)] = k[0]          # many equal keys: stability matters
        keys = torch.from_numpy(k).cuda()
        vals = torch.arange(n, dtype=torch.int32, device="cuda")
        keys_copy, vals_copy = keys.clone(), vals.clone()
        ko_s, vo_s = _sort_static(S, keys, vals, bits)
        ko_r, vo_r = _sort_reference(S, keys, vals, bits)
        torch.cuda.synchronize()
        assert torch.equal(ko_s, ko_r)
        assert torch.equal(vo_s, vo_r)
        assert torch.equal(keys, keys_copy) and torch.equal(vals, vals_copy)   # inputs left intact
        order = np.argsort(k, kind="stable")
        assert np.array_equal(vo_s.cpu().numpy(), order.astype(np.int32))


def test_static_sort_allocates_nothing():
    """After a first call (which loads the library's device code on the
    device), a call leaves the device's free memory and torch's allocator
    statistics unchanged: nothing is allocated or freed."""
    from paper_1812_04719_gb300 import stiv as S
    rng = np.random.default_rng(7)
    n = 200_003
    keys = torch.from_numpy(rng.integers(0, 1 << 40, size=n, dtype=np.int64)).cuda()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    st = torch.cuda.current_stream().cuda_stream
    S.stiv_sort_pairs_static(st, n, 40, keys.data_ptr(), vals.data_ptr(), ko.data_ptr(), vo.data_ptr())
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    S.stiv_sort_pairs_static(st, n, 40, keys.data_ptr(), vals.data_ptr(), ko.data_ptr(), vo.data_ptr())
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for k in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current",
              "allocated_bytes.all.current"):
        assert stats1.get(k, 0) == stats0.get(k, 0), k
    order = np.argsort(keys.cpu().numpy(), kind="stable")
    assert np.array_equal(vo.cpu().numpy(), order.astype(np.int32))


def test_static_sort_rejects_oversize():
    from paper_1812_04719_gb300 import stiv as S
    n = S.SORT_STATIC_MAX + 1
    with pytest.raises(S.StivError):
        # rejected on the host before any pointer is touched
        S.stiv_sort_pairs_static(torch.cuda.current_stream().cuda_stream, n, 8, 16, 16, 16, 16)
