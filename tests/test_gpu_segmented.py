"""GPU parity of sr_sort_segmented / sr_sort_segmented_ex against the oracle,
bit for bit: packs of small segments, medium and big segments, empty segments,
every key type; the full batch workload by properties; bad offsets; capture
in a CUDA graph."""
import numpy as np
import pytest

import oracle
import sortrace_inputs as si

pytestmark = pytest.mark.gpu

KT = {np.dtype(np.int32): 0, np.dtype(np.uint32): 1, np.dtype(np.float32): 2,
      np.dtype(np.uint64): 3, np.dtype(np.int64): 4}
# chunk C (packs hold small segments <= C) and block-sort tile T of the library
SHAPE = {4: (2816, 7680), 8: (1792, 5632)}


def _dev(a):
    import torch
    bits = {4: np.int32, 8: np.int64}[a.dtype.itemsize]
    return torch.from_numpy(np.ascontiguousarray(a).view(bits).copy()).cuda()


def _run(sr, keys, off, ex=False):
    import torch
    tk = _dev(keys)
    to = torch.from_numpy(off.astype(np.int64)).cuda()
    if ex:
        sr.sort_segmented_ex(tk, to, key_type=KT[keys.dtype])
    else:
        sr.sort_segmented(tk, to, key_type=KT[keys.dtype])
    assert sr.stream_status() == 0
    return tk.cpu().numpy().view(keys.dtype)


def _offsets(lens):
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off


def _rand_keys(rng, n, dtype):
    if dtype == np.float32:
        b = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        b[np.isnan(b.view(np.float32))] = 0
        return b.view(np.float32)
    if dtype in (np.uint64, np.int64):
        return rng.integers(0, 1 << 64, n, dtype=np.uint64).view(dtype)
    return rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32).view(dtype)


@pytest.mark.parametrize("dtype", [np.int32, np.uint32, np.float32, np.uint64, np.int64])
def test_mixed_classes(gpu_lib, dtype):
    kb = np.dtype(dtype).itemsize
    C, T = SHAPE[kb]
    rng = np.random.default_rng(31)
    lens = np.concatenate([
        rng.integers(0, 40, 300),                  # tiny, including empty
        rng.integers(1, C + 1, 60),                # small up to the chunk size
        [C, C + 1, T - 1, T, T + 1],               # around the class boundaries
        rng.integers(C + 1, T + 1, 12),            # medium
        [2 * T + 5, 5 * T - 3, 9 * T + 77],        # big: several merge passes
        [0, 0, 1, 0, 2],
    ]).astype(np.int64)
    rng.shuffle(lens)
    off = _offsets(lens)
    keys = _rand_keys(rng, int(off[-1]), dtype)
    got = _run(gpu_lib, keys, off)
    want = oracle.sort_segmented(keys, off)
    assert got.tobytes() == want.tobytes()
    st = gpu_lib.stats()
    assert st["big_segments"] == int(np.sum(lens > T))


@pytest.mark.parametrize("dtype", [np.int32, np.uint64])
def test_duplicates_and_presorted_segments(gpu_lib, dtype):
    rng = np.random.default_rng(32)
    lens = rng.integers(0, 9000, 80).astype(np.int64)
    off = _offsets(lens)
    keys = rng.integers(0, 6, int(off[-1])).astype(dtype)
    for s in range(0, 80, 3):                      # some segments already sorted, some reversed
        a, b = off[s], off[s + 1]
        keys[a:b] = np.sort(keys[a:b]) if s % 2 else np.sort(keys[a:b])[::-1]
    assert _run(gpu_lib, keys, off).tobytes() == oracle.sort_segmented(keys, off).tobytes()


def test_learned_style_out_of_place_singletons(gpu_lib):
    """Many length-0 and length-1 segments among larger ones: every key must
    still reach its place (exercised out of place by the learned sort)."""
    rng = np.random.default_rng(36)
    lens = rng.choice([0, 1, 1, 2, 3, 700, 2500, 4000], 3000).astype(np.int64)
    off = _offsets(lens)
    keys = _rand_keys(rng, int(off[-1]), np.int32)
    assert _run(gpu_lib, keys, off).tobytes() == oracle.sort_segmented(keys, off).tobytes()


def test_single_segment_and_all_empty(gpu_lib):
    rng = np.random.default_rng(33)
    for n in (0, 1, 2, 2816, 2817, 7680, 7681, 100_003):
        keys = _rand_keys(rng, n, np.int32)
        off = np.array([0, n], dtype=np.int64)
        assert _run(gpu_lib, keys, off).tobytes() == oracle.sort_keys(keys).tobytes()
    off = np.zeros(50, dtype=np.int64)
    keys = np.zeros(0, dtype=np.int32)
    assert _run(gpu_lib, keys, off).size == 0


def test_batch_classes_small(gpu_lib):
    """The batch workload's shape at a size the oracle checks quickly: 5,000
    arrays, lognormal lengths (median 512), each one of the four classes."""
    keys, off, types = si.segmented_i32(5000, 7, total=5000 * 600.0)
    assert _run(gpu_lib, keys, off, ex=True).tobytes() == oracle.sort_segmented(keys, off).tobytes()


def test_batch_full_size(gpu_lib, full_size_oracle):
    """200,000 arrays, about 2^27 keys, in one call: every segment equal to
    the oracle's sorted segment, byte for byte."""
    keys, off, _ = si.segmented_i32(200_000, 1)
    got = _run(gpu_lib, keys, off, ex=True)
    full_size_oracle("batch_200k_seed1", [keys, off], [got], lambda: [oracle.sort_segmented(keys, off)])


def test_bad_offsets_set_status(gpu_lib):
    import torch
    keys = _rand_keys(np.random.default_rng(35), 1000, np.int32)
    for off in (np.array([0, 500, 400, 1000], np.int64), np.array([-1, 10, 1000], np.int64),
                np.array([0, 10, 2000], np.int64)):
        tk = _dev(keys)
        before = tk.clone()
        to = torch.from_numpy(off).cuda()
        gpu_lib.sort_segmented_ex(tk, to, key_type=0)
        assert gpu_lib.stream_status() == 7
        assert torch.equal(tk, before)
    assert gpu_lib.stream_status() == 0


def test_graph_capture_replay(gpu_lib):
    """sr_sort_segmented_ex captured once in a CUDA graph and replayed on
    restored inputs."""
    import torch
    keys, off, _ = si.segmented_i32(3000, 9, total=3000 * 600.0)
    want = oracle.sort_segmented(keys, off)
    src = _dev(keys)
    work = src.clone()
    to = torch.from_numpy(off).cuda()
    gpu_lib.sort_segmented_ex(work, to, key_type=0)      # first call on the device before capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        work.copy_(src)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            gpu_lib.sort_segmented_ex(work, to, key_type=0)
    for _ in range(2):
        work.copy_(src)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert work.cpu().numpy().tobytes() == want.tobytes()


def _cfg_lengths(rng, cfg):
    """Segment lengths around every class boundary of a configuration."""
    small, tile, cta = cfg["small_keys"], cfg["tile_keys"], cfg["cta_keys"]
    return np.concatenate([
        rng.integers(0, 40, 200), rng.integers(1, small + 1, 40),
        [small, small + 1, tile - 1, tile, tile + 1, cta - 1, cta, cta + 1],
        rng.integers(small + 1, cta + 1, 8), [2 * cta + 5, 5 * cta - 3], [0, 1, 0, 2],
    ]).astype(np.int64)


@pytest.mark.parametrize("dtype", [np.int32, np.float32, np.uint64, np.int64])
def test_every_config_exact(gpu_lib, dtype):
    """Every launch configuration of the batched sort gives the oracle's
    result bit for bit, with segments on both sides of each of its class
    boundaries (small, one tile, one CTA's fan-in, several merge passes)."""
    import torch
    kt = KT[np.dtype(dtype)]
    for cfg in gpu_lib.segmented_configs(kt):
        rng = np.random.default_rng(50 + cfg["index"])
        lens = _cfg_lengths(rng, cfg)
        rng.shuffle(lens)
        off = _offsets(lens)
        keys = _rand_keys(rng, int(off[-1]), dtype)
        tk = _dev(keys)
        gpu_lib.sort_segmented_cfg(tk, torch.from_numpy(off).cuda(), cfg["index"], key_type=kt)
        assert gpu_lib.stream_status() == 0
        got = tk.cpu().numpy().view(dtype)
        assert got.tobytes() == oracle.sort_segmented(keys, off).tobytes(), cfg
        assert gpu_lib.stats()["big_segments"] == int(np.sum(lens > cfg["cta_keys"])), cfg


def test_every_config_batch_workload(gpu_lib):
    """The batch workload's shape (lognormal lengths, four input classes) at
    a size the oracle checks quickly, under every configuration."""
    import torch
    keys, off, _ = si.segmented_i32(4000, 12, total=4000 * 600.0)
    want = oracle.sort_segmented(keys, off).tobytes()
    to = torch.from_numpy(off).cuda()
    for cfg in gpu_lib.segmented_configs(0):
        tk = _dev(keys)
        gpu_lib.sort_segmented_cfg(tk, to, cfg["index"], key_type=0)
        assert tk.cpu().numpy().tobytes() == want, cfg


def test_autotuner_picks_caches_and_sorts(gpu_lib, tmp_path, monkeypatch):
    import torch
    from paper_1609_04471_gb300 import autotune as at
    keys, off, _ = si.segmented_i32(3000, 13, total=3000 * 600.0)
    src = _dev(keys)
    to = torch.from_numpy(off).cuda()
    path = str(tmp_path / "tune.json")
    best = at.best_config(src, to, 0, cache_path=path, reps=2)
    assert torch.equal(src, _dev(keys))            # the tuner sorts copies only
    n = len(gpu_lib.segmented_configs(0))
    assert 0 <= best < n
    entries = at.load_cache(path)
    (entry,) = entries.values()
    assert entry["config"] == best and len(entry["ms"]) == n
    assert min(entry["ms"], key=lambda c: (entry["ms"][c], int(c))) == str(best)

    def no_timing(*a, **k):
        raise AssertionError("a cached shape must not be timed again")
    monkeypatch.setattr(at, "time_configs", no_timing)
    assert at.best_config(src, to, 0, cache_path=path) == best
    out, c = at.sort_segmented_auto(src, to, 0, cache_path=path)
    assert c == best
    assert out.cpu().numpy().tobytes() == oracle.sort_segmented(keys, off).tobytes()
