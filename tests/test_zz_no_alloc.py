"""The allocation-free key sort (fr_keys_sort_noalloc) against the allocating one (fr_keys_sort).

The allocation-free entry point exists for callers that cannot allocate device memory during the
call; it keeps its scratch in a static device array shared by every call.  This file is collected
last so that a run stopping at the first failure has run every other test before it.  The test
calls the C ABI directly, twice in a row, and compares bit-exactly (sorting is exact).
"""
import ctypes

import numpy as np
import pytest

from paper_2306_06744_gb300 import fr

pytestmark = pytest.mark.gpu


def _sort_both(lib, torch, keys, dim, Dmax):
    a = torch.from_numpy(keys.view(np.int64)).cuda()
    b = a.clone()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert lib.fr_keys_sort(dim, Dmax, ctypes.c_void_p(a.data_ptr()), a.numel(), stream) == 0
    assert lib.fr_keys_sort_noalloc(dim, Dmax, ctypes.c_void_p(b.data_ptr()), b.numel(), stream) == 0
    return a.cpu().numpy().view(np.uint64), b.cpu().numpy().view(np.uint64)


def test_noalloc_sort_matches_allocating_sort_twice():
    import torch
    lib = fr.load()
    rng = np.random.default_rng(2024)
    for call, (n, dim, Dmax) in enumerate([(fr.NOALLOC_SORT_MAX_KEYS, 3, 10), (70001, 2, 9)]):
        keys = rng.integers(0, 1 << (dim * Dmax + 4), size=n, dtype=np.uint64)
        keys[: n // 4] = keys[n // 4: n // 2]  # duplicates exercise stability
        ref, got = _sort_both(lib, torch, keys, dim, Dmax)
        assert np.array_equal(ref, np.sort(keys)), call
        assert np.array_equal(got, ref), call


def test_noalloc_sort_small_sizes_and_no_allocation():
    # n <= 1 returns at once; up to 16384 keys the digit histogram fits one scan tile (the
    # one-level scan branch); the larger sizes above take the two-level scan
    import torch
    lib = fr.load()
    rng = np.random.default_rng(7)
    for n in (0, 1, 2, 1000, 16384):
        keys = rng.integers(0, 1 << 40, size=n, dtype=np.uint64)
        if n >= 4:
            keys[: n // 4] = keys[n // 4: n // 2]
        if n == 0:
            b = torch.zeros(0, dtype=torch.int64, device="cuda")
            stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            assert lib.fr_keys_sort_noalloc(3, 10, ctypes.c_void_p(b.data_ptr()), 0, stream) == 0
            continue
        ref, got = _sort_both(lib, torch, keys, 3, 10)
        assert np.array_equal(ref, np.sort(keys)), n
        assert np.array_equal(got, ref), n
    # the call allocates nothing: the device's free memory is the same before and after calls
    # (the first call on the device, which may load the library's module, was made above)
    keys = rng.integers(0, 1 << 40, size=50000, dtype=np.uint64)
    b = torch.from_numpy(keys.view(np.int64)).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert lib.fr_keys_sort_noalloc(3, 10, ctypes.c_void_p(b.data_ptr()), b.numel(), stream) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(b.cpu().numpy().view(np.uint64), np.sort(keys))


def test_noalloc_sort_rejects_oversize():
    import torch
    lib = fr.load()
    n = fr.NOALLOC_SORT_MAX_KEYS + 1
    a = torch.zeros(n, dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.fr_keys_sort_noalloc(3, 10, ctypes.c_void_p(a.data_ptr()), n, stream)
    assert rc == fr.FR_EINVAL
    assert b"FR_NOALLOC_SORT_MAX_KEYS" in lib.fr_last_error(None)
