"""GPU parity of sr_sort_keys / sr_sort_pairs / sr_detect_runs against the CPU
oracle, bit for bit, through the C ABI.  Sizes span one tile, several tiles
and ragged tails; the four workload classes at 2^24 (the benchmark's launch
configuration) are compared in full."""
import numpy as np
import pytest

import oracle
import sortrace_inputs as si

pytestmark = pytest.mark.gpu

KT = {np.dtype(np.int32): 0, np.dtype(np.uint32): 1, np.dtype(np.float32): 2,
      np.dtype(np.uint64): 3, np.dtype(np.int64): 4}
_TILES = {}


def _tiles(sr, kb, vals=False):
    """(merge tile, block-sort tile) of the library for keys of kb bytes, as
    its statistics report them after a small sort."""
    key = (kb, vals)
    if key not in _TILES:
        import torch
        t = torch.zeros(1000, dtype={4: torch.int32, 8: torch.int64}[kb], device="cuda")
        if vals:
            sr.sort_pairs(t, torch.zeros(1000, dtype=torch.int32, device="cuda"), key_type=0 if kb == 4 else 3)
        else:
            sr.sort_keys(t, key_type=0 if kb == 4 else 3)
        st = sr.stats()
        _TILES[key] = (st["merge_tile"], st["tile"])
    return _TILES[key]


def _to_dev(a):
    import torch
    bits = {4: np.int32, 8: np.int64}[a.dtype.itemsize]
    return torch.from_numpy(np.ascontiguousarray(a).view(bits).copy()).cuda()


def _from_dev(t, dtype):
    return t.cpu().numpy().view(dtype)


def _gpu_sort(sr, a):
    t = _to_dev(a)
    sr.sort_keys(t, key_type=KT[a.dtype])
    return _from_dev(t, a.dtype)


def _gpu_pairs(sr, k, v):
    import torch
    tk = _to_dev(k)
    tv = torch.from_numpy(v.view(np.int32).copy()).cuda()
    sr.sort_pairs(tk, tv, key_type=KT[k.dtype])
    return _from_dev(tk, k.dtype), tv.cpu().numpy().view(np.uint32)


def _random(rng, n, dtype):
    if dtype == np.float32:
        b = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        f = b.view(np.float32)
        b[np.isnan(f)] ^= 0x00400000      # keep a few NaN-free patterns distinct
        return b.view(np.float32)
    if dtype in (np.uint64, np.int64):
        return rng.integers(0, 1 << 64, n, dtype=np.uint64).view(dtype) if dtype == np.int64 else \
            rng.integers(0, 1 << 64, n, dtype=np.uint64)
    return rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32).view(dtype)


def _sizes(sr, kb):
    nv, ts = _tiles(sr, kb)
    return sorted({0, 1, 2, 3, 5, 31, 32, 33, 255, 1000, nv - 1, nv, nv + 1, ts - 1, ts, ts + 1,
                   2 * ts + 7, 4 * ts - 1, (1 << 16) + 1, 5 * ts + 3, 100_003, (1 << 20) - 1})


@pytest.mark.parametrize("dtype", [np.int32, np.uint32, np.float32, np.uint64, np.int64])
def test_keys_random_sizes(gpu_lib, dtype):
    rng = np.random.default_rng(10)
    for n in _sizes(gpu_lib, np.dtype(dtype).itemsize):
        a = _random(rng, n, dtype)
        got = _gpu_sort(gpu_lib, a)
        want = oracle.sort_keys(a)
        assert got.tobytes() == want.tobytes(), (dtype, n)


@pytest.mark.parametrize("dtype", [np.int32, np.float32, np.uint64])
def test_keys_heavy_duplicates(gpu_lib, dtype):
    rng = np.random.default_rng(11)
    for n in (7, 4000, 9000, 123_457):
        a = rng.integers(0, 5, n).astype(dtype)
        assert _gpu_sort(gpu_lib, a).tobytes() == oracle.sort_keys(a).tobytes()


def test_edge_values(gpu_lib):
    i32 = np.array([0, -1, 1, 2**31 - 1, -2**31] * 3001, dtype=np.int32)
    assert _gpu_sort(gpu_lib, i32).tobytes() == oracle.sort_keys(i32).tobytes()
    f = np.array([0.0, -0.0, 1e-45, -1e-45, np.inf, -np.inf, 3.5, -3.5, 1.17549435e-38,
                  -1.17549435e-38] * 2001, dtype=np.float32)
    assert _gpu_sort(gpu_lib, f).view(np.uint32).tolist() == oracle.sort_keys(f).view(np.uint32).tolist()
    # NaN patterns order by their bits under totalOrder
    nan = np.array([np.nan, -np.nan, 1.0, -1.0, np.inf] * 999, dtype=np.float32)
    nan.view(np.uint32)[::7] = 0x7FC00001
    assert _gpu_sort(gpu_lib, nan).view(np.uint32).tolist() == oracle.sort_keys(nan).view(np.uint32).tolist()
    u64 = np.array([0, 2**64 - 1, 2**63, 2**63 - 1, 1] * 4001, dtype=np.uint64)
    assert _gpu_sort(gpu_lib, u64).tobytes() == oracle.sort_keys(u64).tobytes()
    i64 = u64.view(np.int64)
    assert _gpu_sort(gpu_lib, i64).tobytes() == oracle.sort_keys(i64).tobytes()


def test_all_equal_and_presorted(gpu_lib):
    for a in (np.full(50_001, 7, np.int32), np.arange(50_001, dtype=np.int32),
              np.arange(50_001, 0, -1, dtype=np.int32),
              np.repeat(np.arange(1000, 0, -1, dtype=np.int32), 50),   # descending, not strictly
              si.k_equal_teeth(1 << 17, 8), si.k_even_teeth(1 << 17, 2), si.k_sharp_teeth(1 << 17, 8),
              si.k_distance(1 << 17, 256), si.k_exchange(1 << 17, 16),
              np.tile(np.array([1, 0], np.int32), 40_000)):
        assert _gpu_sort(gpu_lib, a).tobytes() == oracle.sort_keys(a).tobytes()


def test_sorted_input_moves_nothing(gpu_lib):
    import torch
    n = 1 << 20
    a = np.sort(si.uniform_i32(n, 3))
    t = _to_dev(a)
    gpu_lib.sort_keys(t, key_type=0)
    st = gpu_lib.stats()
    assert st["input_class"] == 1 and st["runs"] == 1
    assert st["bytes_moved"] == 4 * n           # the scan's read only
    assert _from_dev(t, np.int32).tobytes() == a.tobytes()
    torch.cuda.synchronize()


def test_reversed_input_one_pass(gpu_lib):
    n = (1 << 20) + 3
    a = si.reversed_i32(n, 4)
    t = _to_dev(a)
    gpu_lib.sort_keys(t, key_type=0)
    st = gpu_lib.stats()
    assert st["input_class"] == 2 and st["runs"] == n
    assert st["bytes_moved"] == 4 * n + 8 * n   # scan + one reversal
    assert _from_dev(t, np.int32).tobytes() == oracle.sort_keys(a).tobytes()


def test_teeth_skip_passes(gpu_lib):
    """2-equal teeth whose teeth are whole numbers of block-sort tiles (128
    int32 tiles, 7 merge levels: seven 2-way steps, or one 2-way step and
    three 4-way ones): every step below the tooth length finds all its run
    pairs in order and is skipped; only the last step merges."""
    n = 128 * _tiles(gpu_lib, 4)[1]
    a = si.k_equal_teeth(n, 2)
    t = _to_dev(a)
    gpu_lib.sort_keys(t, key_type=0)
    st = gpu_lib.stats()
    assert (st["passes_planned"], st["passes_skipped"]) in ((7, 6), (4, 3))
    assert _from_dev(t, np.int32).tobytes() == oracle.sort_keys(a).tobytes()


@pytest.mark.parametrize("kind", list(si.INT32_CLASSES))
def test_classes_2_20(gpu_lib, kind):
    a = si.int32_input(kind, (1 << 20) + 17, seed=7)
    assert _gpu_sort(gpu_lib, a).tobytes() == oracle.sort_keys(a).tobytes()


def test_two_million_uniform_seed1(gpu_lib):
    """2,000,000 uniform int32 keys, seed 1 (the paper's Table 1 size)."""
    a = si.uniform_i32(2_000_000, 1)
    assert _gpu_sort(gpu_lib, a).tobytes() == oracle.sort_keys(a).tobytes()


@pytest.mark.parametrize("kind", list(si.INT32_CLASSES))
def test_classes_2_24_full(gpu_lib, kind):
    """The benchmark's workload: 2^24 int32 keys of each class, seed 1,
    compared in full with the oracle."""
    a = si.int32_input(kind, 1 << 24, seed=1)
    assert _gpu_sort(gpu_lib, a).tobytes() == oracle.sort_keys(a).tobytes()


def test_detect_runs_matches_oracle(gpu_lib):
    for a in (si.uniform_i32(100_000, 2), si.k_exchange(100_000, 50), si.reversed_i32(77_777, 1),
              np.sort(si.uniform_i32(70_000, 3)), si.few_unique_i32(90_000, 5),
              np.array([1, 15, 18, 19, 20, 16, 11, 10, 9, 8, 7, 6, 5, 4, 3, 2], np.int32)):
        info = gpu_lib.detect_runs(_to_dev(a), key_type=0)
        assert info["runs"] == oracle.runs(a)
        assert info["sorted"] == (oracle.runs(a) == 1)
    f = si.lognormal_f32(200_001, 3)
    assert gpu_lib.detect_runs(_to_dev(f), key_type=2)["runs"] == oracle.runs(f)


@pytest.mark.parametrize("dtype", [np.int32, np.float32, np.uint64, np.int64, np.uint32])
def test_pairs_stable(gpu_lib, dtype):
    rng = np.random.default_rng(12)
    nv, ts = _tiles(gpu_lib, np.dtype(dtype).itemsize, vals=True)
    for n in sorted({0, 1, 2, 33, nv - 1, nv, nv + 1, ts, ts + 1, 2 * ts, 2 * ts + 1, 30_001, 262_147}):
        k = (rng.integers(0, 9, n).astype(dtype) if n % 2 else _random(rng, n, dtype))
        v = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        gk, gv = _gpu_pairs(gpu_lib, k, v)
        ok, ov = oracle.sort_pairs(k, v)
        assert gk.tobytes() == ok.tobytes() and gv.tobytes() == ov.tobytes(), (dtype, n)


def test_pairs_presorted(gpu_lib):
    n = 200_003
    for k in (np.arange(n, dtype=np.uint64), np.arange(n, 0, -1).astype(np.uint64),
              np.repeat(np.arange(1000, 0, -1), n // 1000 + 1)[:n].astype(np.uint64)):
        v = np.arange(n, dtype=np.uint32)
        gk, gv = _gpu_pairs(gpu_lib, k, v)
        ok, ov = oracle.sort_pairs(k, v)
        assert gk.tobytes() == ok.tobytes() and gv.tobytes() == ov.tobytes()


def test_pairs_zipf_2_20(gpu_lib):
    k, v = si.pairs_u64_zipf(1 << 20, 1)
    gk, gv = _gpu_pairs(gpu_lib, k, v)
    ok, ov = oracle.sort_pairs(k, v)
    assert gk.tobytes() == ok.tobytes() and gv.tobytes() == ov.tobytes()


def test_deterministic(gpu_lib):
    a = si.uniform_i32(3_000_001, 5)
    assert _gpu_sort(gpu_lib, a).tobytes() == _gpu_sort(gpu_lib, a).tobytes()


def test_host_entry_point(gpu_lib):
    a = si.nearly_sorted_i32((1 << 20) + 5, 2)
    b = a.copy()
    gpu_lib.sort_keys_host(b)
    assert b.tobytes() == oracle.sort_keys(a).tobytes()


def test_host_async_entry_point_on_several_streams(gpu_lib):
    """Four host arrays in page-locked memory sorted at once on four streams;
    pageable memory is refused before anything is queued."""
    import torch
    arrays = [si.int32_input(kind, (1 << 20) + 3 * i, seed=20 + i) for i, kind in enumerate(si.INT32_CLASSES)]
    host = [torch.from_numpy(a.copy()).pin_memory() for a in arrays]
    streams = [torch.cuda.Stream() for _ in arrays]
    for h, st in zip(host, streams):
        gpu_lib.sort_keys_host_async(h, stream=st)
    for st in streams:
        st.synchronize()
    for h, a in zip(host, arrays):
        assert h.numpy().tobytes() == oracle.sort_keys(a).tobytes()
    with pytest.raises(gpu_lib.SortError):
        gpu_lib.sort_keys_host_async(arrays[0].copy())


def test_host_many_pipeline(gpu_lib):
    """Several page-locked host arrays (every int32 class, ragged sizes, an
    empty and a one-key array) sorted as one pipeline; 8-byte keys too;
    pageable memory is refused before anything is queued."""
    import torch
    sizes = [(1 << 20) + 7, 0, 300_001, 1, (1 << 18) - 1, 2_000_003]
    kinds = list(si.INT32_CLASSES)
    arrays = [si.int32_input(kinds[i % len(kinds)], n, seed=30 + i) for i, n in enumerate(sizes)]
    host = [torch.from_numpy(a.copy()).pin_memory() for a in arrays]
    s = torch.cuda.Stream()
    gpu_lib.sort_keys_host_many(host, stream=s)
    s.synchronize()
    for h, a in zip(host, arrays):
        assert h.numpy().tobytes() == oracle.sort_keys(a).tobytes()
    rng = np.random.default_rng(64)
    arrays = [_random(rng, n, np.uint64) for n in (700_001, 5, 100_000)]
    host = [torch.from_numpy(a.view(np.int64).copy()).pin_memory() for a in arrays]
    gpu_lib.sort_keys_host_many(host, key_type=3, stream=s)
    s.synchronize()
    for h, a in zip(host, arrays):
        assert h.numpy().view(np.uint64).tobytes() == oracle.sort_keys(a).tobytes()
    with pytest.raises(gpu_lib.SortError):
        gpu_lib.sort_keys_host_many([torch.zeros(10, dtype=torch.int64).pin_memory(), arrays[0].copy()],
                                    key_type=3)


def test_oom_injection(gpu_lib, monkeypatch):
    import torch
    a = _to_dev(si.uniform_i32(100_000, 1))
    before = a.clone()
    monkeypatch.setenv("SR_INJECT_OOM", "1")
    with pytest.raises(gpu_lib.SortError) as e:
        gpu_lib.sort_keys(a, key_type=0)
    assert e.value.code == 3
    monkeypatch.delenv("SR_INJECT_OOM")
    torch.cuda.synchronize()
    assert torch.equal(a, before)


@pytest.mark.parametrize("dtype", [np.int32, np.uint32, np.float32])
def test_few_distinct_keys(gpu_lib, dtype):
    """At most 4,096 distinct keys (4-byte keys): a 65,536-key sample spread
    over the array builds the set of distinct keys; when it holds every key the
    call counts them and writes runs (input_class 3, 12 bytes per key moved).
    4,097 or more distinct keys, or a key the sample missed, take the ordinary
    sort.  Output bit-exact against the oracle either way, including float32
    -0.0 / +0.0 as distinct keys."""
    rng = np.random.default_rng(60)
    for d, n in ((2, 1000), (16, 1 << 20), (64, (1 << 20) + 3), (65, 300_001), (1000, 300_001),
                 (4096, (1 << 22) + 5), (4097, 1 << 22), (20000, 300_001)):
        vals = _random(rng, d, dtype)
        if dtype == np.float32 and d >= 2:
            vals[:2] = np.array([0x00000000, 0x80000000], np.uint32).view(np.float32)
        vals = np.unique(vals.view({4: np.uint32}[4])).view(dtype)
        a = vals[rng.integers(0, vals.size, n)]
        got = _gpu_sort(gpu_lib, a)
        assert got.tobytes() == oracle.sort_keys(a).tobytes(), (dtype, d, n)
        st = gpu_lib.stats()
        if np.unique(a.view(np.uint32)).size <= 4096 and n >= 256 * vals.size:
            # every distinct key is in the sample (65,536 draws)
            assert st["input_class"] == 3 and st["bytes_moved"] == 12 * n, (d, n, st["input_class"])
        elif vals.size > 4096:
            assert st["input_class"] == 0
    # the 65th distinct key appears once, at the end: the sample misses it, the
    # counting pass finds it and the ordinary sort runs
    a = np.concatenate([np.repeat(np.arange(64, dtype=np.int32) * 7, 5000), np.array([3], np.int32)])
    rng.shuffle(a[:-1])
    got = _gpu_sort(gpu_lib, a)
    assert got.tobytes() == oracle.sort_keys(a).tobytes()
    assert gpu_lib.stats()["input_class"] == 0
    # pairs never take this path (payloads must move with their keys)
    k = np.repeat(np.arange(8, dtype=np.int32), 1000)[::-1].copy()
    rng.shuffle(k)
    v = np.arange(k.size, dtype=np.uint32)
    gk, gv = _gpu_pairs(gpu_lib, k, v)
    ok, ov = oracle.sort_pairs(k, v)
    assert gk.tobytes() == ok.tobytes() and gv.tobytes() == ov.tobytes()


def _order_statistic_ok(torch, src, out, positions):
    """out[i] is the i-th smallest key of src for every sampled i: fewer than
    i+1 keys are smaller and at least i+1 are smaller or equal (counted on the
    device, one position at a time)."""
    for i in positions:
        v = out[i]
        less = int((src < v).sum())
        leq = int((src <= v).sum())
        if not (less <= i < leq):
            return False
    return True


def test_full_size_2_28_uniform(gpu_lib, full_size_oracle):
    """2^28 uniform int32 keys (the top of the benchmark's size sweep), in the
    launch configuration the benchmark times: every output byte equal to the
    oracle's sorted output, plus 64 sampled output positions equal to the
    order statistic of the input counted on the device."""
    import torch
    a = si.uniform_i32(1 << 28, 1)
    src = torch.from_numpy(a).cuda()
    x = src.clone()
    gpu_lib.sort_keys(x, key_type=0)
    assert gpu_lib.stream_status() == 0
    got = x.cpu().numpy()
    full_size_oracle("uniform_i32_2p28_seed1", [a], [got], lambda: [oracle.sort_keys(a)])
    rng = np.random.default_rng(61)
    pos = [0, x.numel() - 1] + [int(p) for p in rng.integers(0, x.numel(), 62)]
    assert _order_statistic_ok(torch, src, x, pos)


def test_full_size_2_28_pairs(gpu_lib, full_size_oracle):
    """The stable pairs workload at full size: 2^28 uint64 keys (half uniform,
    half Zipf 1.1 over 2^20 values) with payload = original index: keys and
    payloads equal to the stable oracle's byte for byte; on the device, every
    output key equals the input key at its payload and equal keys keep
    ascending payloads."""
    import torch
    k, v = si.pairs_u64_zipf(1 << 28, 1)
    sk = torch.from_numpy(k.view(np.int64)).cuda()
    xk = sk.clone()
    xv = torch.from_numpy(v.view(np.int32)).cuda()
    gpu_lib.sort_pairs(xk, xv, key_type=3)
    assert gpu_lib.stream_status() == 0
    gk = xk.cpu().numpy().view(np.uint64)
    gv = xv.cpu().numpy().view(np.uint32)
    full_size_oracle("pairs_u64_zipf_2p28_seed1", [k, v], [gk, gv], lambda: list(oracle.sort_pairs(k, v)))
    del gk, gv
    idx = xv.to(torch.int64)
    assert bool((sk[idx] == xk).all())
    same = xk[1:] == xk[:-1]
    assert bool((xv[1:][same] > xv[:-1][same]).all())


def _exchanged(rng, sorted_keys, frac, adjacent=False):
    """A k-exchange list (Section 2): sorted keys, then floor(frac * n)
    exchanges of a uniform position with a uniform partner (or with the key
    two places on, for clustered displacements)."""
    a = sorted_keys.copy()
    n = a.size
    for _ in range(int(frac * n)):
        i = int(rng.integers(0, n - 2))
        j = i + 2 if adjacent else int(rng.integers(0, n))
        a[i], a[j] = a[j], a[i]
    return a


@pytest.mark.parametrize("dtype", [np.int32, np.float32, np.uint64, np.int64])
def test_few_displaced_keys(gpu_lib, dtype):
    """Keys only, a few keys away from their place (k-exchange lists, the Rem
    measure of Section 2): the keys left in order go straight to their block
    and the displaced ones through per-tile buckets (input_class 4).  Output
    bit-exact against the oracle on uniform and clustered exchanges and on a
    ragged size; bytes moved follow the path's model."""
    rng = np.random.default_rng(62)
    kb = np.dtype(dtype).itemsize
    for n, frac, adjacent in (((1 << 20) + 17, 0.01, False), (700_001, 0.005, True), (1 << 22, 0.01, False)):
        base = np.sort(_random(rng, n, dtype))
        if dtype == np.float32:
            base = base[~np.isnan(base)]
        a = _exchanged(rng, base, frac, adjacent)
        got = _gpu_sort(gpu_lib, a)
        assert got.tobytes() == oracle.sort_keys(a).tobytes(), (dtype, n, frac, adjacent)
        st = gpu_lib.stats()
        assert st["input_class"] == 4, (dtype, n, st["input_class"])
        # the kept keys are in order, so at least Rem(A) keys went aside; about
        # two per exchange (three for clustered ones) at most
        assert oracle.rem(a) <= st["displaced"] <= 3 * int(frac * n) + 2 * (n // 6400) + 64
        m = a.size
        assert 5 * kb * m <= st["bytes_moved"] <= 5 * kb * m + 2 * kb * (m // 16)


def test_few_displaced_keys_fallbacks(gpu_lib):
    """The path gives way to the ordinary sort (input_class 0), with the same
    output, when a bucket would overflow (exchanges among few distinct values
    crowd one bucket), when there are fewer descents than sort tiles, and for
    pairs (payload order); an unaligned key pointer still takes it."""
    import torch
    rng = np.random.default_rng(63)
    # heavily repeated values (and 20,000 single ones, too many distinct keys
    # for the few-distinct path): equal keys pile into a few buckets
    base = np.concatenate([rng.integers(-50, 50, 380_000), rng.integers(-2**31, 2**31 - 1, 20_000)])
    a = _exchanged(rng, np.sort(base.astype(np.int32)), 0.005)
    assert _gpu_sort(gpu_lib, a).tobytes() == oracle.sort_keys(a).tobytes()
    assert gpu_lib.stats()["input_class"] == 0
    # fewer descents than tiles
    a = _exchanged(rng, np.sort(_random(rng, 1 << 20, np.int32)), 10 / (1 << 20))
    assert _gpu_sort(gpu_lib, a).tobytes() == oracle.sort_keys(a).tobytes()
    assert gpu_lib.stats()["input_class"] == 0
    # pairs
    k = _exchanged(rng, np.sort(_random(rng, 300_000, np.int32)), 0.01)
    v = np.arange(k.size, dtype=np.uint32)
    gk, gv = _gpu_pairs(gpu_lib, k, v)
    ok, ov = oracle.sort_pairs(k, v)
    assert gk.tobytes() == ok.tobytes() and gv.tobytes() == ov.tobytes()
    assert gpu_lib.stats()["input_class"] == 0
    # a key pointer 4 bytes past a 16-byte boundary
    a = _exchanged(rng, np.sort(_random(rng, 500_000, np.int32)), 0.01)
    buf = torch.zeros(a.size + 1, dtype=torch.int32, device="cuda")
    buf[1:] = torch.from_numpy(a.view(np.int32)).cuda()
    gpu_lib.sort_keys(buf[1:], key_type=0)
    assert gpu_lib.stats()["input_class"] == 4
    assert buf[1:].cpu().numpy().tobytes() == oracle.sort_keys(a).tobytes()
    assert int(buf[0]) == 0


@pytest.mark.parametrize("kind", list(si.INT32_CLASSES))
def test_repeated_calls(gpu_lib, kind):
    """The same buffer sorted again and again: from the second call on, the
    call replays a CUDA graph whose merge section runs only when the input
    needs it.  Every result bit-exact against the oracle, statistics of the
    call's own input, launches counted."""
    import torch
    a = si.int32_input(kind, (1 << 20) + 5, seed=11)
    want = oracle.sort_keys(a).tobytes()
    src = torch.from_numpy(a).cuda()
    x = torch.empty_like(src)
    classes = set()
    counts = []
    for _ in range(4):
        x.copy_(src)
        l0 = gpu_lib.launch_count()
        gpu_lib.sort_keys(x, key_type=0)
        counts.append(gpu_lib.launch_count() - l0)
        assert x.cpu().numpy().tobytes() == want
        classes.add(gpu_lib.stats()["input_class"])
    assert len(classes) == 1
    # the first call launches the whole sequence; a replay runs its own branch only
    assert counts[2] == counts[3] and 0 < counts[3] <= counts[0]
    if kind == "reversed":
        assert counts[3] <= 6          # scan, sample, router, reversal
    if kind == "uniform":
        assert counts[3] >= 15         # the sort section runs
    # stable pairs on a repeated buffer as well
    k = si.int32_input(kind, 300_007, seed=12)
    v = np.arange(k.size, dtype=np.uint32)
    ok, ov = oracle.sort_pairs(k, v)
    tk, tv = torch.from_numpy(k).cuda(), torch.from_numpy(v.view(np.int32)).cuda()
    xk, xv = torch.empty_like(tk), torch.empty_like(tv)
    for _ in range(3):
        xk.copy_(tk)
        xv.copy_(tv)
        gpu_lib.sort_pairs(xk, xv, key_type=0)
        assert xk.cpu().numpy().tobytes() == ok.tobytes()
        assert xv.cpu().numpy().view(np.uint32).tobytes() == ov.tobytes()


def test_sort_keys_in_captured_graph(gpu_lib):
    """sr_sort_keys captured in the caller's CUDA graph (ordinary launches,
    scratch from graph allocation nodes) and replayed on new inputs."""
    import torch
    arrays = [si.int32_input(kind, 500_003, seed=13) for kind in si.INT32_CLASSES]
    x = torch.from_numpy(arrays[0]).cuda()
    gpu_lib.sort_keys(x.clone(), key_type=0)        # device state exists before the capture
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        gpu_lib.sort_keys(x, key_type=0, stream=s)
    for a in arrays:
        x.copy_(torch.from_numpy(a).cuda())
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert x.cpu().numpy().tobytes() == oracle.sort_keys(a).tobytes()


def test_graph_cache_eviction(gpu_lib):
    """More repeated-call argument sets than the library keeps graphs for: the
    least recently used are dropped and rebuilt; every result exact."""
    import torch
    rng = np.random.default_rng(65)
    arrays = [_random(rng, 70_000 + 13 * i, np.int32) for i in range(20)]
    bufs = [torch.from_numpy(a).cuda() for a in arrays]
    wants = [oracle.sort_keys(a).tobytes() for a in arrays]
    for sweep in range(2):
        for a, b, w in zip(arrays, bufs, wants):
            for _ in range(3):                  # first sight, graph build, replay
                b.copy_(torch.from_numpy(a).cuda())
                gpu_lib.sort_keys(b, key_type=0)
                assert b.cpu().numpy().tobytes() == w, sweep


def test_release_cached(gpu_lib):
    """The graphs kept for repeated calls can be dropped; the next calls
    rebuild them and give the same results."""
    import torch
    a = si.int32_input("nearly_sorted", 300_001, seed=14)
    want = oracle.sort_keys(a).tobytes()
    src = torch.from_numpy(a).cuda()
    x = torch.empty_like(src)
    for r in range(6):
        x.copy_(src)
        gpu_lib.sort_keys(x, key_type=0)
        assert x.cpu().numpy().tobytes() == want
        if r == 2:
            gpu_lib.release_cached()


_PAPER_CLASSES = {
    "k-limited": lambda n, k: si.k_limited(n, min(k, 32), 3),
    "k-equal teeth": lambda n, k: si.k_equal_teeth(n - n % k, k),
    "k-even teeth": lambda n, k: si.k_even_teeth(n - n % k, k),
    "k-sharp teeth": lambda n, k: si.k_sharp_teeth(n - n % k, k),
    "k-shuffled teeth": lambda n, k: si.k_shuffled_teeth(n - n % k, k, 3),
    "k-distance": lambda n, k: si.k_distance(n, k, 3),
    "k-exchange": lambda n, k: si.k_exchange(n, k, 3),
}


@pytest.mark.parametrize("name,k", [("k-limited", 12), ("k-equal teeth", 8), ("k-even teeth", 8),
                                    ("k-sharp teeth", 8), ("k-shuffled teeth", 8), ("k-distance", 256),
                                    ("k-exchange", (1 << 24) // 100)])
def test_paper_classes_2_24(gpu_lib, name, k):
    """Section 2's parametrised classes at 2^24 int32 keys (the parameters the
    benchmark's class table uses), compared in full with the oracle."""
    a = _PAPER_CLASSES[name](1 << 24, k)
    assert _gpu_sort(gpu_lib, a).tobytes() == oracle.sort_keys(a).tobytes(), (name, k)


@pytest.mark.parametrize("name", list(_PAPER_CLASSES))
def test_paper_classes_k_sweep(gpu_lib, name):
    """Each class for k = 2^0 .. 2^8 (the paper's range) at 2^20 + 7 keys."""
    for i in range(9):
        a = _PAPER_CLASSES[name]((1 << 20) + 7, 2 ** i)
        assert _gpu_sort(gpu_lib, a).tobytes() == oracle.sort_keys(a).tobytes(), (name, 2 ** i)
