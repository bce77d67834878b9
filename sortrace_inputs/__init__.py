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

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "_gen.c")
_LIB = os.path.join(_HERE, "_build", "libsr_gen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the multi-threaded fills (_gen.c) with gcc."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-Wall", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _c():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, sz, vp = ctypes.c_uint64, ctypes.c_size_t, ctypes.c_void_p
            lib.sg_key.argtypes = [u64, u64]
            lib.sg_key.restype = u64
            lib.sg_stream.argtypes = [u64, u64, vp, sz]
            lib.sg_lognormal.argtypes = [u64, u64, u64, vp, vp, vp, ctypes.c_int, vp, sz]
            lib.sg_zipf_pairs.argtypes = [u64, u64, u64, vp, sz, vp, sz, sz, vp, vp, vp]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags keep the draws of different purposes independent
_STREAMS = {
    "uniform": 1, "reversed": 2, "nearly": 3, "nearly_swap": 4, "few": 5,
    "few_pick": 6, "u64": 7, "zipf_table": 8, "zipf_u": 9, "shuffle": 10,
    "lognormal_c": 11, "lognormal_u1": 12, "lognormal_u2": 13, "seg_len_u1": 14,
    "seg_len_u2": 15, "seg_type": 16, "teeth": 17, "kdist": 18, "kexch": 19,
    "klimited": 20, "kshuffle": 21,
}


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: str) -> int:
    """key = mix(seed * golden + tag) of a named stream (64-bit wrap-around)."""
    tag = _STREAMS[stream]
    with np.errstate(over="ignore"):
        return int(_mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN + np.uint64(tag)],
                                 dtype=np.uint64))[0])


def u64_stream(seed: int, stream: str, count: int, offset: int = 0) -> np.ndarray:
    """``count`` SplitMix64 outputs of stream ``stream`` starting at counter
    ``offset``: out[i] = mix(key + (offset + i + 1) * golden), where
    key = mix(seed * golden + tag)."""
    key = _key(seed, stream)
    if count >= (1 << 16):
        out = np.empty(count, dtype=np.uint64)
        _c().sg_stream(key, offset, _ptr(out), count)
        return out
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix(np.uint64(key) + ctr * _GOLDEN)


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


def zipf_table(seed: int = 1, support: int = 1 << 20) -> np.ndarray:
    """``support`` distinct random uint64 values in a seeded order; rank r maps
    to table[r - 1]."""
    table = np.unique(u64_stream(seed, "zipf_table", support + support // 8))
    if table.size < support:
        raise RuntimeError("zipf value table has too many collisions")
    order = np.argsort(u64_stream(seed, "zipf_table", table.size, offset=1 << 40), kind="stable")
    return table[order[:support]]


def pairs_u64_zipf(n: int, seed: int = 1, s: float = 1.1, support: int = 1 << 20):
    """uint64 keys, half uniform and half Zipf(s) over ``support`` distinct
    random values, in uniformly random order; payload = original index.

    n // 2 positions get uniform keys and the rest Zipf keys (rank by inverse
    CDF on the cumulative table, in double); the Zipf positions are a
    uniformly random subset of exactly that size (selection sampling, Knuth's
    Algorithm S).  As every key is an independent draw, this is the two halves
    concatenated and shuffled uniformly."""
    nu = n // 2
    nz = n - nu
    table = zipf_table(seed, support)
    cdf = zipf_cdf(s, support)
    keys = np.empty(n, dtype=np.uint64)
    vals = np.empty(n, dtype=np.uint32)
    flags = np.empty(n, dtype=np.uint8)
    _c().sg_zipf_pairs(_key(seed, "shuffle"), _key(seed, "u64"), _key(seed, "zipf_u"), _ptr(cdf), support,
                       _ptr(table), n, nz, _ptr(keys), _ptr(vals), _ptr(flags))
    return keys, vals


# ------------------------------------------------------- float32 lognormal

LOGNORMAL_MIX = ((0.0, 0.5, 0.5), (2.0, 1.0, 0.3), (5.0, 0.3, 0.2))  # (mu, sigma, weight)


def lognormal_f32(n: int, seed: int = 1, mix=LOGNORMAL_MIX) -> np.ndarray:
    """float32 keys from a lognormal mixture: pick a component by its weight,
    then x = exp(mu + sigma*z), z standard normal by Box-Muller (double), then
    round to float32.  All keys are positive and finite."""
    mu = np.array([m[0] for m in mix], dtype=np.float64)
    sg = np.array([m[1] for m in mix], dtype=np.float64)
    w = np.cumsum([m[2] for m in mix])
    cumw = (w / w[-1]).astype(np.float64)
    out = np.empty(n, dtype=np.float32)
    if n:
        _c().sg_lognormal(_key(seed, "lognormal_c"), _key(seed, "lognormal_u1"), _key(seed, "lognormal_u2"),
                          _ptr(mu), _ptr(sg), _ptr(cumw), len(mix), _ptr(out), n)
    return out


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
    Each array follows its type's class, drawn from per-type streams indexed
    by the global key position: uniform; strictly descending distinct values;
    ascending distinct values with floor(0.01 len) exchanges; 16 values."""
    lens = segment_lengths(num, seed, **kw)
    types = _below(u64_stream(seed, "seg_type", num), 4)
    off = np.zeros(num + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    n = int(off[-1])
    keys = np.empty(n, dtype=np.int32)
    seg = np.repeat(np.arange(num, dtype=np.int64), lens)
    t = types[seg]
    pos = np.nonzero(t == 0)[0]
    keys[pos] = (u64_stream(seed * 7919 + 1, "uniform", n)[pos] >> np.uint64(32)).astype(np.uint32).view(np.int32)
    pos = np.nonzero(t == 3)[0]
    vals = few_unique_values(seed * 7919 + 2)
    keys[pos] = vals[_below(u64_stream(seed * 7919 + 2, "few_pick", n)[pos], 16)]
    for ty, stream in ((1, "reversed"), (2, "nearly")):
        pos = np.nonzero(t == ty)[0]
        if pos.size == 0:
            continue
        s_of = seg[pos]
        L = lens[s_of]
        i = pos - off[s_of]
        q = (np.int64(1) << 32) // L
        r = _below(u64_stream(seed * 7919 + 3 + ty, stream, n)[pos], np.minimum(q, (1 << 32) - 1))
        r = np.where(q > 1, r, 0)
        j = (L - 1 - i) if ty == 1 else i
        keys[pos] = (-(1 << 31) + j * q + r).astype(np.int32)
    # nearly sorted: floor(0.01 len) exchanges inside each such array, in order
    near = np.nonzero(types == 2)[0]
    m = np.floor(0.01 * lens[near]).astype(np.int64)
    tot = int(m.sum())
    if tot:
        u = u64_stream(seed * 7919 + 5, "nearly_swap", 2 * tot)
        segs = np.repeat(near, m)
        base = off[segs]
        Ls = lens[segs]
        ii = base + _below(u[0::2], Ls)
        jj = base + _below(u[1::2], Ls)
        _apply_swaps(keys, ii, jj)
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


def k_limited(n: int, k: int, seed: int = 1) -> np.ndarray:
    """n values drawn uniformly from 2^k distinct ones, 0 .. 2^k - 1 (Section 2;
    the blow-up map is monotone and omitted)."""
    return (u64_stream(seed, "klimited", n) >> np.uint64(64 - k)).astype(np.int32) if k > 0 else \
        np.zeros(n, np.int32)


def k_shuffled_teeth(n: int, k: int, seed: int = 1) -> np.ndarray:
    """k-sharp teeth whose k sections are interleaved into one sequence at
    random, each section keeping its own order (Section 2)."""
    L = n // k
    sections = k_sharp_teeth(L * k, k).reshape(k, L)
    labels = np.repeat(np.arange(k), L)
    order = np.argsort(u64_stream(seed, "kshuffle", L * k), kind="stable")
    labels = labels[order]
    out = np.empty(L * k, np.int32)
    out[np.argsort(labels, kind="stable")] = sections.reshape(-1)   # section j's positions, in order
    return out


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
