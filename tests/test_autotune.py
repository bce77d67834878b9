"""Host logic of the batched sort's autotuner: workload keys, the cache file
and the choice of the fastest configuration (no GPU)."""
import json

import numpy as np

from paper_1609_04471_gb300 import autotune as at


def test_workload_key_bands():
    lens = np.array([0, 512, 600, 500, 3000])
    k = at.workload_key("GPU X", 0, 4612, lens)
    # 4612 keys -> band 13 (2^12 <= x < 2^13); 5 segments -> band 3; median of the
    # non-empty lengths 556 -> band 10
    assert k == "GPU X|kt0|n13|s3|m10"
    assert at.workload_key("GPU X", 0, 4612, np.zeros(4, np.int64)) == "GPU X|kt0|n13|s3|m0"
    assert at.workload_key("GPU X", 3, 4612, lens) != k


def test_select_best_ties_to_lower_index():
    assert at.select_best({0: 2.0, 1: 1.5, 2: 1.5, 3: 9.0}) == 1
    assert at.select_best({4: 0.1}) == 4


def test_cache_round_trip_and_version(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert at.load_cache(p) == {}
    at.save_cache(p, {"a": {"config": 2, "ms": {"0": 1.0, "2": 0.5}}})
    assert at.load_cache(p)["a"]["config"] == 2
    with open(p, "w") as f:
        json.dump({"version": 999, "entries": {"a": {"config": 1}}}, f)
    assert at.load_cache(p) == {}                  # another format: ignored
    with open(p, "w") as f:
        f.write("not json")
    assert at.load_cache(p) == {}


def test_cache_path_from_environment(monkeypatch, tmp_path):
    monkeypatch.setenv(at.CACHE_ENV, str(tmp_path / "x.json"))
    assert at.default_cache_path() == str(tmp_path / "x.json")
