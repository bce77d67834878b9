"""GPU parity, bit for bit against the oracle, for inputs holding the largest
key of their type.  The block sort and the 2-way merge tiles mark the end of
every run with the largest order image and merge with one comparison per step
only when no key equals that mark; a tile or window holding such keys takes
the bounded merge steps instead.  These inputs put the largest key (int32
2^31 - 1, uint32 2^32 - 1, the float32 bit pattern 0x7fffffff whose order
image is the largest, the int64 and uint64 maxima) in some tiles and windows
and not in others, at sizes spanning many tiles with ragged tails, for keys
alone and for stable pairs (equal keys keep their input order)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

KT = {np.dtype(np.int32): 0, np.dtype(np.uint32): 1, np.dtype(np.float32): 2,
      np.dtype(np.uint64): 3, np.dtype(np.int64): 4}
TOP = {np.dtype(np.int32): np.int32(2 ** 31 - 1), np.dtype(np.uint32): np.uint32(2 ** 32 - 1),
       np.dtype(np.float32): np.uint32(0x7FFFFFFF).view(np.float32),
       np.dtype(np.uint64): np.uint64(2 ** 64 - 1), np.dtype(np.int64): np.int64(2 ** 63 - 1)}


def _input(rng, n, dtype, share, alphabet):
    """Keys of `dtype`: a fraction `share` equal to the type's largest key, the
    rest random (full range, or `alphabet` values, many ties)."""
    dt = np.dtype(dtype)
    if alphabet:
        a = rng.integers(0, alphabet, n).astype(np.uint64)
    else:
        a = rng.integers(0, 2 ** 63, n, dtype=np.uint64) * 2 + rng.integers(0, 2, n, dtype=np.uint64)
    if dt.itemsize == 4:
        a = (a & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        if dt == np.float32:
            a[(a & 0x7F800000) == 0x7F800000] = 0x3F800000     # no NaN or infinity from the random bits
        a = a.view(dt)
    else:
        a = a.view(dt)
    a = a.copy()
    top = rng.random(n) < share
    a[top] = TOP[dt]
    return a


def _dev(a):
    import torch
    bits = {4: np.int32, 8: np.int64}[a.dtype.itemsize]
    return torch.from_numpy(np.ascontiguousarray(a).view(bits).copy()).cuda()


@pytest.mark.parametrize("dtype", [np.int32, np.uint32, np.float32, np.uint64, np.int64])
def test_keys_with_the_largest_key(gpu_lib, dtype):
    rng = np.random.default_rng(17)
    for n in (1000, 16896 * 3 + 11, 12800 * 5 + 3, 200_003, (1 << 20) + 77):
        for share, alphabet in ((0.0, None), (1e-4, None), (0.01, None), (0.3, 9), (1.0, None)):
            a = _input(rng, n, dtype, share, alphabet)
            x = _dev(a)
            gpu_lib.sort_keys(x, key_type=KT[np.dtype(dtype)])
            got = x.cpu().numpy().view(a.dtype)
            assert got.tobytes() == oracle.sort_keys(a).tobytes(), (dtype, n, share, alphabet)
    assert gpu_lib.stream_status() == 0


@pytest.mark.parametrize("dtype", [np.int32, np.uint64])
def test_pairs_with_the_largest_key(gpu_lib, dtype):
    import torch
    rng = np.random.default_rng(19)
    for n in (12800 * 2 + 5, 16896 * 2 + 7, 200_003, (1 << 20) + 3):
        for share, alphabet in ((1e-3, None), (0.2, 5)):
            k = _input(rng, n, dtype, share, alphabet)
            v = np.arange(n, dtype=np.uint32)
            xk = _dev(k)
            xv = torch.from_numpy(v.view(np.int32).copy()).cuda()
            gpu_lib.sort_pairs(xk, xv, key_type=KT[np.dtype(dtype)])
            ok, ov = oracle.sort_pairs(k, v)
            assert xk.cpu().numpy().view(k.dtype).tobytes() == ok.tobytes(), (dtype, n, share)
            assert xv.cpu().numpy().view(np.uint32).tobytes() == ov.tobytes(), (dtype, n, share)
    assert gpu_lib.stream_status() == 0
