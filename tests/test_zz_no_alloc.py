"""The allocation-free sort entry point (mpm_radix_sort_pairs_noalloc).

It serves callers that may not allocate device memory -- an engine that owns
every allocation and offers no allocator hook, or a real-time frame callback
where an allocation could stall the device.  The test calls it through the C
ABI twice in a row (the second call on a different, smaller input, so stale
scratch from the first call must not leak into the result) and checks each
result against the allocating entry point mpm_radix_sort_pairs and against
numpy's stable argsort: a sort is integer work, so both comparisons are
bit-exact.  This file is collected last on purpose so a failure here cannot
hide any other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2111_00699_gb300 import _lib, build
    build.build()
    assert torch.cuda.is_available(), "GPU test"
    return _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _reference_sort(L, keys, vals, bits):
    """The existing entry point, with its scratch allocated by the caller."""
    n = keys.numel()
    nb = ctypes.c_size_t()
    assert L.load().mpm_radix_sort_pairs(None, None, None, None, n, bits, None, ctypes.byref(nb), None) == 0
    scratch = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    ko, vo = torch.empty_like(keys), torch.empty_like(vals)
    st = L.load().mpm_radix_sort_pairs(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), n, bits, _ptr(scratch),
                                       ctypes.byref(nb), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    return ko, vo


def _inputs(seed, n, bits):
    rng = np.random.default_rng(seed)
    k = rng.integers(0, min(1 << bits, max(2, n // 3)), size=n, dtype=np.uint64)
    k = ((k * np.uint64(2654435761)) % np.uint64(1 << bits)).astype(np.uint32)
    return (torch.from_numpy(k.view(np.int32)).cuda(),
            torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda())


def test_noalloc_sort_matches_allocating_sort_twice(lib):
    L = lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed, n, bits in ((1, lib.SORT_NOALLOC_MAX_KEYS, 24), (2, 123_457, 30)):
        keys, vals = _inputs(seed, n, bits)
        ko = torch.full_like(keys, -1)
        vo = torch.full_like(vals, -1)
        st = L.mpm_radix_sort_pairs_noalloc(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), n, bits, stream)
        assert st == lib.MPM_OK
        rk, rv = _reference_sort(lib, keys, vals, bits)
        torch.cuda.synchronize()
        assert torch.equal(ko, rk) and torch.equal(vo, rv)
        # and, independently of the library's sort code, against numpy's stable sort
        k_in = keys.cpu().numpy().view(np.uint32)
        idx = np.argsort(k_in, kind="stable")
        np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32), k_in[idx])
        np.testing.assert_array_equal(vo.cpu().numpy(), vals.cpu().numpy()[idx])


def test_noalloc_sort_rejects_oversize_input(lib):
    L = lib.load()
    n = lib.SORT_NOALLOC_MAX_KEYS + 1
    # nothing is launched for an oversize request, so null pointers are safe here
    assert L.mpm_radix_sort_pairs_noalloc(None, None, None, None, n, 24, None) == lib.MPM_ECAPACITY
    assert L.mpm_radix_sort_pairs_noalloc(None, None, None, None, 0, 24, None) == lib.MPM_OK
