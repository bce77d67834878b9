"""sr_sort_keys_noalloc, the entry point for callers that must not allocate
device memory (its scratch is a fixed array inside the library).  Checked
through the C ABI against sr_sort_keys, bit for bit, on calls made back to back
so that each call starts from the previous call's leftover scratch.  This file
is collected last so a failure here cannot hide earlier results."""
import ctypes

import numpy as np
import pytest

import sortrace_inputs as si

pytestmark = pytest.mark.gpu

MAX_KEYS = 1 << 20


def _dev(a):
    import torch
    bits = {4: np.int32, 8: np.int64}[a.dtype.itemsize]
    return torch.from_numpy(np.ascontiguousarray(a).view(bits).copy()).cuda()


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_sort_keys_back_to_back(gpu_lib):
    import torch
    lib = gpu_lib.load()
    cases = [
        (si.uniform_i32(MAX_KEYS, 21), 0),                      # the largest size allowed
        (si.nearly_sorted_i32(MAX_KEYS - 3, 22), 0),            # ragged tail, leftovers from above
        (si.lognormal_f32(300_001, 23), 2),
        (si.reversed_i32(99_999, 24), 0),
        (np.random.default_rng(25).integers(0, 1 << 64, 700_001, dtype=np.uint64), 3),
        # 8-byte keys at exactly the largest size allowed (the widest layout)
        (np.random.default_rng(29).integers(0, 1 << 64, MAX_KEYS, dtype=np.uint64), 3),
        (np.random.default_rng(30).integers(-(1 << 63), (1 << 63) - 1, MAX_KEYS, dtype=np.int64), 4),
        (np.random.default_rng(26).integers(0, 9, 5000).astype(np.int64), 4),
        (si.few_unique_i32(7_681, 27).view(np.uint32), 1),
    ]
    for a, kt in cases:
        ref = _dev(a)
        got = _dev(a)
        assert lib.sr_sort_keys(ctypes.c_void_p(ref.data_ptr()), a.size, kt, _stream()) == 0
        for _ in range(2):                                      # two calls in a row
            got.copy_(_dev(a))
            assert lib.sr_sort_keys_noalloc(ctypes.c_void_p(got.data_ptr()), a.size, kt, _stream()) == 0
            torch.cuda.synchronize()
            assert torch.equal(got, ref), (a.dtype, a.size, kt)


def test_noalloc_rejects_too_many_keys(gpu_lib):
    import torch
    lib = gpu_lib.load()
    x = _dev(si.uniform_i32(MAX_KEYS + 1, 28))
    before = x.clone()
    assert lib.sr_sort_keys_noalloc(ctypes.c_void_p(x.data_ptr()), MAX_KEYS + 1, 0, _stream()) == 1
    torch.cuda.synchronize()
    assert torch.equal(x, before)
