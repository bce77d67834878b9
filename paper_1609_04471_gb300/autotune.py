"""Autotuner for the batched (segmented) sort.

The segmented sort has a small list of launch configurations per key width
(strategy for small segments, CTA size, keys per thread of packs and of
block-sort tiles, merge fan-in; see sr_segmented_config_info).  All give the
same result; which is fastest depends on the mix of segment lengths.  The
tuner times every configuration on the caller's batch (a copy of it, with
CUDA events on the current stream), keeps the fastest, and caches the choice
in a JSON file keyed by the GPU, the key type and a coarse description of the
workload (total keys, segment count and median segment length, each as a
power-of-two band), so later batches of the same shape skip the timing.

The cache lives in $SORTRACE_TUNE_CACHE, else ~/.cache/sortrace_gb300/
segmented.json.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

CACHE_ENV = "SORTRACE_TUNE_CACHE"
CACHE_VERSION = 1


def default_cache_path() -> str:
    p = os.environ.get(CACHE_ENV)
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "sortrace_gb300", "segmented.json")


def _band(x: float) -> int:
    """Power-of-two band of a non-negative quantity (0 for x < 1)."""
    return 0 if x < 1 else int(math.floor(math.log2(x))) + 1


def workload_key(gpu: str, key_type: int, n_keys: int, lengths) -> str:
    """Cache key of a batch: GPU name, key type, and the bands of the total
    key count, the segment count and the median non-empty segment length."""
    import numpy as np
    lengths = np.asarray(lengths)
    nz = lengths[lengths > 0]
    med = float(np.median(nz)) if nz.size else 0.0
    return f"{gpu}|kt{key_type}|n{_band(n_keys)}|s{_band(lengths.size)}|m{_band(med)}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return {}
    if not isinstance(d, dict) or d.get("version") != CACHE_VERSION:
        return {}
    return d.get("entries", {})


def save_cache(path: str, entries: dict) -> None:
    """Writes the cache atomically (a temporary file renamed over the old)."""
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune-", suffix=".json")
    with os.fdopen(fd, "w") as f:
        json.dump({"version": CACHE_VERSION, "entries": entries}, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def select_best(timings: dict) -> int:
    """The configuration with the smallest time; ties go to the lower index."""
    if not timings:
        raise ValueError("no timings")
    return min(timings, key=lambda c: (timings[c], c))


def time_configs(keys, offsets, key_type: int | None = None, reps: int = 3, warmup: int = 1,
                 configs=None) -> dict:
    """Milliseconds of sr_sort_segmented_cfg for each configuration on a copy
    of `keys` (the input itself is not changed): the minimum over `reps`
    timed calls after `warmup` untimed ones, CUDA events on the current
    stream, the copy restored before every call."""
    import torch
    from . import segmented_configs, sort_segmented_cfg, key_type_of, stream_status
    kt = key_type_of(keys) if key_type is None else key_type
    idx = [c["index"] for c in segmented_configs(kt)] if configs is None else list(configs)
    work = torch.empty_like(keys)
    out = {}
    for c in idx:
        best = float("inf")
        for r in range(warmup + reps):
            work.copy_(keys)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sort_segmented_cfg(work, offsets, c, key_type=kt)
            e1.record()
            e1.synchronize()
            if r >= warmup:
                best = min(best, e0.elapsed_time(e1))
        if stream_status() != 0:
            raise RuntimeError(f"segmented sort reported status {stream_status()} under configuration {c}")
        out[c] = best
    return out


def best_config(keys, offsets, key_type: int | None = None, cache_path: str | None = None,
                retune: bool = False, reps: int = 3) -> int:
    """The cached configuration for this batch's shape, timing every
    configuration (and caching the winner) on a miss or when `retune`."""
    import torch
    from . import key_type_of
    kt = key_type_of(keys) if key_type is None else key_type
    off = offsets.cpu().numpy()
    lengths = off[1:] - off[:-1]
    gpu = torch.cuda.get_device_name(keys.device)
    key = workload_key(gpu, kt, keys.numel(), lengths)
    path = cache_path or default_cache_path()
    entries = load_cache(path)
    if not retune and key in entries:
        return int(entries[key]["config"])
    t = time_configs(keys, offsets, kt, reps=reps)
    best = select_best(t)
    entries = load_cache(path)                     # another process may have written meanwhile
    entries[key] = {"config": best, "ms": {str(c): round(v, 4) for c, v in t.items()}}
    save_cache(path, entries)
    return best


def sort_segmented_auto(keys, offsets, key_type: int | None = None, stream=None,
                        cache_path: str | None = None):
    """sort_segmented_ex under the tuned configuration for this batch's
    shape; returns (keys, config)."""
    from . import sort_segmented_cfg
    c = best_config(keys, offsets, key_type, cache_path=cache_path)
    sort_segmented_cfg(keys, offsets, c, key_type=key_type, stream=stream)
    return keys, c
