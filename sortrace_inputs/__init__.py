"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the smoke check and the benchmark.  It holds
no sorting arithmetic: it only draws numbers.  Every draw comes from one
counter-based generator, SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated on the counter
``i`` of a named stream, so the bytes depend only on (seed, stream, i) and are
the same on every machine.

Input classes (Section 2 of the paper, and the workload descriptions):

* ``uniform_i32``      random items over the whole int32 range.
* ``reversed_i32``     reversely sorted, strictly descending, distinct values.
* ``nearly_sorted_i32`` ascending, then m = floor(0.01 n) exchanges of a random
  position with a random partner (a k-exchange list with k = m).
* ``few_unique_i32``   values drawn uniformly from 16 distinct random int32s
  (the "few unique" class; the paper builds it as a k-limited list).
* ``pairs_u64_zipf``   uint64 keys: half uniform, half Zipf(s = 1.1) ranks over
  2^20 distinct random values, shuffled; payload = original index.
* ``lognormal_f32``    float32 from the 3-component lognormal mixture.
* ``segment_lengths``  lognormal lengths, median 512, clipped to [1, 2^20].
* ``teeth`` / ``k_distance`` / ``k_exchange`` classes of Section 2 on small n,
  for the run-detection tests.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags keep the draws of different purposes independent
_STREAMS = {
    "uniform": 1, "reversed": 2, "nearly": 3, "nearly_swap": 4, "few": 5,
    "few_pick": 6, "u64": 7, "zipf_table": 8, "zipf_u": 9, "shuffle": 10,
    "lognormal_c": 11, "lognormal_u1": 12, "lognormal_u2": 13, "seg_len_u1": 14,
    "seg_len_u2": 15, "seg_type": 16, "teeth": 17, "kdist": 18, "kexch": 19,
}


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def u64_stream(seed: int, stream: str, count: int, offset: int = 0) -> np.ndarray:
    """``count`` SplitMix64 outputs of stream ``stream`` starting at counter
    ``offset``: out[i] = mix(key + (offset + i + 1) * golden), where
    key = mix(seed * golden + tag)."""
    tag = _STREAMS[stream]
    with np.errstate(over="ignore"):
        key = _mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN + np.uint64(tag)],
                            dtype=np.uint64))[0]
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix(key + ctr * _GOLDEN)


def _below(u: np.ndarray, m) -> np.ndarray:
    """Maps uint64 draws to integers in [0, m) (multiply-shift on the top 32
    bits; m may be an array).  m must be < 2^32."""
    hi = u >> np.uint64(32)
    with np.errstate(over="ignore"):
        return ((hi * np.asarray(m, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)


def _unit(u: np.ndarray) -> np.ndarray:
    """uint64 draws -> doubles in [0, 1) from the top 53 bits."""
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ------------------------------------------------------------- int32 classes

def uniform_i32(n: int, seed: int = 1) -> np.ndarray:
    return (u64_stream(seed, "uniform", n) >> np.uint64(32)).astype(np.uint32).view(np.int32)


def _spread_i32(n: int, seed: int, stream: str) -> np.ndarray:
    """n distinct int32 values in ascending order: INT32_MIN + i*q + r_i,
    q = floor(2^32 / n), r_i uniform in [0, q)."""
    if n == 0:
        return np.zeros(0, np.int32)
    q = (1 << 32) // n
    r = _below(u64_stream(seed, stream, n), min(q, (1 << 32) - 1)) if q > 1 else np.zeros(n, np.int64)
    v = -(1 << 31) + np.arange(n, dtype=np.int64) * q + r
    return v.astype(np.int32)


def reversed_i32(n: int, seed: int = 1) -> np.ndarray:
    """Strictly descending, distinct (reversely sorted)."""
    return _spread_i32(n, seed, "reversed")[::-1].copy()


def nearly_sorted_i32(n: int, seed: int = 1, frac: float = 0.01) -> np.ndarray:
    """Ascending distinct values, then floor(frac*n) exchanges of a uniform
    position with a uniform partner (a k-exchange list, Section 2)."""
    a = _spread_i32(n, seed, "nearly")
    m = int(math.floor(frac * n))
    if m and n > 1:
        u = u64_stream(seed, "nearly_swap", 2 * m)
        ij = _below(u, n)
        _apply_swaps(a, ij[0::2], ij[1::2])
    return a


def _apply_swaps(a: np.ndarray, ii: np.ndarray, jj: np.ndarray) -> None:
    """Applies the exchanges (ii[k], jj[k]) in order k = 0, 1, ..."""
    for i, j in zip(ii.tolist(), jj.tolist()):
        a[i], a[j] = a[j], a[i]


def few_unique_values(seed: int = 1, k: int = 16) -> np.ndarray:
    """k distinct random int32 values (duplicates are redrawn)."""
    vals: list[int] = []
    off = 0
    while len(vals) < k:
        u = int(u64_stream(seed, "few", 1, off)[0] >> np.uint64(32))
        off += 1
        v = u - (1 << 32) if u >= (1 << 31) else u
        if v not in vals:
            vals.append(v)
    return np.array(vals, dtype=np.int32)


def few_unique_i32(n: int, seed: int = 1, k: int = 16) -> np.ndarray:
    vals = few_unique_values(seed, k)
    return vals[_below(u64_stream(seed, "few_pick", n), k)]


INT32_CLASSES = {
    "uniform": uniform_i32,
    "reversed": reversed_i32,
    "nearly_sorted": nearly_sorted_i32,
    "few_unique": few_unique_i32,
}


def int32_input(kind: str, n: int, seed: int = 1) -> np.ndarray:
    return INT32_CLASSES[kind](n, seed)


# ------------------------------------------------------- uint64 key + payload

def zipf_cdf(s: float = 1.1, support: int = 1 << 20) -> np.ndarray:
    """Cumulative Zipf(s) probabilities over ranks 1..support (double)."""
    w = np.arange(1, support + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def pairs_u64_zipf(n: int, seed: int = 1, s: float = 1.1, support: int = 1 << 20):
    """uint64 keys: the first half uniform, the second half Zipf(s) ranks over
    ``support`` distinct random uint64 values (rank r -> table[r-1]); the two
    halves are then shuffled together by a seeded random permutation.  The
    payload is the original index 0..n-1 (uint32)."""
    nu = n // 2
    nz = n - nu
    uni = u64_stream(seed, "u64", nu)
    table = np.unique(u64_stream(seed, "zipf_table", support + support // 8))
    if table.size < support:
        raise RuntimeError("zipf value table has too many collisions")
    # a seeded subset of distinct values, in a seeded order
    order = np.argsort(u64_stream(seed, "zipf_table", table.size, offset=1 << 40), kind="stable")
    table = table[order[:support]]
    cdf = zipf_cdf(s, support)
    ranks = np.searchsorted(cdf, _unit(u64_stream(seed, "zipf_u", nz)), side="right")
    ranks = np.minimum(ranks, support - 1)
    keys = np.concatenate([uni, table[ranks]])
    perm = np.argsort(u64_stream(seed, "shuffle", n), kind="stable")
    keys = keys[perm]
    vals = np.arange(n, dtype=np.uint32)
    return keys, vals


# ------------------------------------------------------- float32 lognormal

LOGNORMAL_MIX = ((0.0, 0.5, 0.5), (2.0, 1.0, 0.3), (5.0, 0.3, 0.2))  # (mu, sigma, weight)


def lognormal_f32(n: int, seed: int = 1, mix=LOGNORMAL_MIX) -> np.ndarray:
    """float32 keys from a lognormal mixture: pick a component by its weight,
    then x = exp(mu + sigma*z), z standard normal by Box-Muller (double), then
    round to float32.  All keys are positive and finite."""
    c = _unit(u64_stream(seed, "lognormal_c", n))
    w = np.cumsum([m[2] for m in mix])
    comp = np.searchsorted(w / w[-1], c, side="right")
    comp = np.minimum(comp, len(mix) - 1)
    mu = np.array([m[0] for m in mix])[comp]
    sg = np.array([m[1] for m in mix])[comp]
    u1 = _unit(u64_stream(seed, "lognormal_u1", n))
    u2 = _unit(u64_stream(seed, "lognormal_u2", n))
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    return np.exp(mu + sg * z).astype(np.float32)


# ------------------------------------------------------- segmented batches

SEG_TYPES = ("uniform", "reversed", "nearly_sorted", "few_unique")


def segment_lengths(num: int, seed: int = 1, median: float = 512.0,
                    total: float = float(1 << 27), max_len: int = 1 << 20) -> np.ndarray:
    """Lognormal lengths with the given median; sigma is chosen so the expected
    total is ``total``: sigma = sqrt(2 ln(total / (num * median))).  Rounded to
    nearest and clipped to [1, max_len]."""
    ratio = total / (num * median)
    sigma = math.sqrt(2.0 * math.log(ratio)) if ratio > 1.0 else 0.0
    u1 = _unit(u64_stream(seed, "seg_len_u1", num))
    u2 = _unit(u64_stream(seed, "seg_len_u2", num))
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    L = np.rint(median * np.exp(sigma * z))
    return np.clip(L, 1, max_len).astype(np.int64)


def segmented_i32(num: int, seed: int = 1, **kw):
    """A batch of ``num`` int32 arrays stored back to back: returns
    (keys, offsets[num+1] int64, types[num] in 0..3 indexing SEG_TYPES).
    Each array is drawn from its type's class with a seed derived from the
    batch seed and the array's index."""
    lens = segment_lengths(num, seed, **kw)
    types = _below(u64_stream(seed, "seg_type", num), 4)
    off = np.zeros(num + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    keys = np.empty(int(off[-1]), dtype=np.int32)
    for t, kind in enumerate(SEG_TYPES):
        idx = np.nonzero(types == t)[0]
        if idx.size == 0:
            continue
        if kind in ("uniform", "few_unique"):
            # one long draw, cut into the arrays of this type
            tot = int(lens[idx].sum())
            sub = (uniform_i32(tot, seed * 7919 + 1) if kind == "uniform"
                   else few_unique_i32(tot, seed * 7919 + 2))
            pos = 0
            for s in idx.tolist():
                L = int(lens[s])
                keys[off[s]:off[s] + L] = sub[pos:pos + L]
                pos += L
        else:
            for s in idx.tolist():
                L = int(lens[s])
                sub_seed = (seed << 20) + s
                keys[off[s]:off[s] + L] = (reversed_i32(L, sub_seed) if kind == "reversed"
                                           else nearly_sorted_i32(L, sub_seed))
    return keys, off, types


# ------------------------------------------- Section 2 presorted classes (tests)

def k_equal_teeth(n: int, k: int) -> np.ndarray:
    """k sorted sections 1..n/k each (Section 2; n divisible by k); the
    blow-up map is omitted: it is monotone and does not change the order."""
    L = n // k
    return np.tile(np.arange(1, L + 1, dtype=np.int32), k)


def k_even_teeth(n: int, k: int) -> np.ndarray:
    """k-equal teeth with the odd-numbered sections (1st, 3rd, ...) reversed."""
    L = n // k
    a = k_equal_teeth(n, k).reshape(k, L)
    a[0::2] = a[0::2, ::-1]
    return a.reshape(-1).copy()


def k_sharp_teeth(n: int, k: int) -> np.ndarray:
    """1..n in k equal sections with the odd-numbered sections reversed."""
    L = n // k
    a = np.arange(1, n + 1, dtype=np.int32).reshape(k, L)
    a[0::2] = a[0::2, ::-1]
    return a.reshape(-1).copy()


def k_distance(n: int, k: int, seed: int = 1) -> np.ndarray:
    """1..n cut into sections of k+1 items, each section shuffled."""
    a = np.arange(1, n + 1, dtype=np.int32)
    L = k + 1
    u = u64_stream(seed, "kdist", n)
    for s in range(0, n, L):
        e = min(n, s + L)
        order = np.argsort(u[s:e], kind="stable")
        a[s:e] = a[s:e][order]
    return a


def k_exchange(n: int, k: int, seed: int = 1) -> np.ndarray:
    """1..n with k exchanges of two random positions."""
    a = np.arange(1, n + 1, dtype=np.int32)
    ij = _below(u64_stream(seed, "kexch", 2 * k), n)
    _apply_swaps(a, ij[0::2], ij[1::2])
    return a
