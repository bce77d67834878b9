"""A plain model of the few-displaced-keys path of the key sort (the keys kept
in order per tile by value bounds, the rest through per-tile buckets), run on
the CPU: it checks that the path's steps give the sorted list for ANY bounds
the medians produce, including adversarial inputs, and that the inputs it is
meant for send few keys to the buckets.  The GPU kernels are compared with
the oracle in tests/test_gpu_sort.py; this pins the algorithm itself."""
import numpy as np
import pytest

import sortrace_inputs as si

CAP = 512          # keys per bucket before the path gives way to the ordinary sort
ROUNDS = 8         # descent-removal rounds per tile


def _model(a, tile=6400, cap=CAP):
    """Returns (sorted output or None if a bucket overflows, displaced count)."""
    u = (a.view(np.uint32) ^ np.uint32(0x80000000)).astype(np.int64)   # order images
    n = u.size
    tiles = (n + tile - 1) // tile
    # bounds: median of the 9 keys around each tile start (positions past the end
    # read the last key), made nondecreasing by a running maximum; bound[0] = 0
    bound = np.zeros(tiles, np.int64)
    for b in range(1, tiles):
        pos = np.minimum(np.arange(b * tile - 4, b * tile + 5), n - 1)
        bound[b] = np.sort(u[pos])[4]
    bound = np.maximum.accumulate(bound)
    slots, buckets = [], [[] for _ in range(tiles)]
    for b in range(tiles):
        x = u[b * tile:min(n, (b + 1) * tile)]
        top = b == tiles - 1
        keep = (x >= bound[b]) & (top | (x < (bound[b + 1] if not top else 0)))
        for r in range(ROUNDS + 1):
            idx = np.nonzero(keep)[0]
            desc = np.nonzero(x[idx][:-1] > x[idx][1:])[0]
            if desc.size == 0:
                break
            if r == ROUNDS:
                keep[:] = False
                break
            keep[idx[desc]] = False
            keep[idx[desc + 1]] = False
        s = x[keep]
        assert np.all(s[:-1] <= s[1:])                       # kept keys are sorted
        assert s.size == 0 or (s[0] >= bound[b] and (top or s[-1] < bound[b + 1]))
        slots.append(s)
        for v in x[~keep]:                                     # the bucket of v's value range
            buckets[int(np.searchsorted(bound, v, side="right")) - 1].append(v)
    if max(len(bk) for bk in buckets) > cap:
        return None, None
    out = np.concatenate([np.sort(np.concatenate([slots[b], np.array(buckets[b], np.int64)]))
                          for b in range(tiles)])
    displaced = sum(len(bk) for bk in buckets)
    return (out ^ 0x80000000).astype(np.uint32).view(np.int32), displaced


def _exchanged(rng, a, m, adjacent=False):
    a = a.copy()
    for _ in range(m):
        i = int(rng.integers(0, a.size - 2))
        j = i + 2 if adjacent else int(rng.integers(0, a.size))
        a[i], a[j] = a[j], a[i]
    return a


@pytest.mark.parametrize("n,frac,adjacent", [(1 << 18, 0.01, False), (200_003, 0.005, True), (300_000, 0.02, False)])
def test_model_sorts_k_exchange_lists(n, frac, adjacent):
    rng = np.random.default_rng(70)
    a = _exchanged(rng, np.sort(rng.integers(-2**31, 2**31 - 1, n).astype(np.int32)), int(frac * n), adjacent)
    out, displaced = _model(a)
    assert out is not None and np.array_equal(out, np.sort(a))
    # about the exchanged keys: two per exchange, three for a clustered one (both
    # ends of each of its two descents), a few more per tile boundary
    assert displaced <= 3 * int(frac * n) + 2 * (n // 6400) + 64


def test_model_on_the_benchmark_class():
    a = si.nearly_sorted_i32(1 << 18, 3)
    out, displaced = _model(a)
    assert np.array_equal(out, np.sort(a)) and displaced < (1 << 18) // 32


def test_model_gives_way_on_crowded_buckets():
    """Exchanges among few distinct values: tiles whose bounds coincide keep
    nothing and their keys crowd one bucket, so the ordinary sort must run."""
    rng = np.random.default_rng(71)
    a = _exchanged(rng, np.sort(rng.integers(-50, 50, 200_000).astype(np.int32)), 500)
    out, _ = _model(a)
    assert out is None


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_model_any_bounds_give_the_sorted_list(seed):
    """Random inputs and few-valued inputs (never sent down the path, their
    bounds are arbitrary) still come out sorted once the buckets may hold
    them: the result never depends on the bounds."""
    rng = np.random.default_rng(seed)
    for a in (rng.integers(-2**31, 2**31 - 1, 20_000).astype(np.int32),
              rng.integers(-3, 3, 20_000).astype(np.int32), si.k_sharp_teeth(20_000, 5)):
        out, _ = _model(a, tile=64, cap=a.size)
        assert out is not None and np.array_equal(out, np.sort(a))
