"""CPU oracle for the sort -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it and the
two share no code; the only module both sides use is ``sortrace_inputs`` (the
seeded input generators, which hold no sort arithmetic).

What it computes (the plain definitions the GPU path must reproduce bit for
bit):

* keys:       the non-decreasing permutation of the input under the key order
              (signed int32/int64, unsigned uint32/uint64, IEEE-754 totalOrder
              for float32).  The result is unique.
* pairs:      the stable sort: ordered by key, equal keys in input order.
* segmented:  every segment [off[s], off[s+1]) sorted on its own.

Implementations (``sr_oracle.c``, plain single-threaded C over the paper's
qsort-style interface):

* ``merge``  natural mergesort with the techniques of the paper's mer6
             (Section 3); ``merge5`` the same without short-run growth (mer5).
* ``quick``  the hybrid quicksort hyb2 (Section 4).
* ``isort``  insertion sort, the brute-force definition.

Also Run(A), Mono(A) and Inv(A) of Section 2, a comparison counter and a trace
of what each merge did (for the worked example of Section 3).

The learned partitioner's model (forward and backward in float64) lives in
``oracle/model.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sr_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsr_oracle.so")
_lock = threading.Lock()
_lib = None

KEY_TYPES = {np.dtype(np.int32): 0, np.dtype(np.uint32): 1, np.dtype(np.float32): 2,
             np.dtype(np.uint64): 3, np.dtype(np.int64): 4}
ALGOS = {"merge": 0, "quick": 1, "isort": 2, "merge5": 3}


def build(force: bool = False) -> str:
    """Compiles sr_oracle.c into a shared library with gcc (plain -O2, no
    machine-specific flags, so x86 and Arm builds agree)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, sz, i32, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64
            lib.sro_sort_keys.argtypes = [vp, sz, i32, i32]
            lib.sro_sort_pairs.argtypes = [vp, vp, sz, i32, i32]
            lib.sro_sort_segmented.argtypes = [vp, vp, sz, i32, i32]
            for f in (lib.sro_runs, lib.sro_mono, lib.sro_inversions, lib.sro_rem):
                f.argtypes = [vp, sz, i32]
                f.restype = u64
            lib.sro_cmp_count.restype = u64
            lib.sro_trace_enable.argtypes = [i32]
            lib.sro_trace_read.argtypes = [vp, i32]
            lib.sro_trace_read.restype = i32
            _lib = lib
    return _lib


def _kt(a: np.ndarray) -> int:
    try:
        return KEY_TYPES[a.dtype]
    except KeyError:
        raise TypeError(f"unsupported key dtype {a.dtype}") from None


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def sort_keys(keys: np.ndarray, algo: str = "merge") -> np.ndarray:
    """Returns a sorted copy of ``keys``."""
    out = np.ascontiguousarray(keys).copy()
    rc = _load().sro_sort_keys(_ptr(out), out.size, _kt(out), ALGOS[algo])
    if rc:
        raise RuntimeError(f"oracle sort failed ({rc})")
    return out


def sort_pairs(keys: np.ndarray, vals: np.ndarray, algo: str = "merge"):
    """Returns (keys, vals) sorted stably by key."""
    k = np.ascontiguousarray(keys).copy()
    v = np.ascontiguousarray(vals, dtype=np.uint32).copy()
    if k.size != v.size:
        raise ValueError("keys and vals differ in length")
    rc = _load().sro_sort_pairs(_ptr(k), _ptr(v), k.size, _kt(k), ALGOS[algo])
    if rc:
        raise RuntimeError(f"oracle pair sort failed ({rc})")
    return k, v


def sort_segmented(keys: np.ndarray, offsets: np.ndarray, algo: str = "merge") -> np.ndarray:
    """Returns a copy of ``keys`` with every segment sorted on its own."""
    k = np.ascontiguousarray(keys).copy()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    if off.size < 1 or off[0] != 0 or off[-1] != k.size:
        raise ValueError("offsets must run from 0 to len(keys)")
    rc = _load().sro_sort_segmented(_ptr(k), _ptr(off), off.size - 1, _kt(k), ALGOS[algo])
    if rc:
        raise RuntimeError(f"oracle segmented sort failed ({rc})")
    return k


def runs(a: np.ndarray) -> int:
    """Run(A): number of descents + 1 (0 for the empty array)."""
    a = np.ascontiguousarray(a)
    return int(_load().sro_runs(_ptr(a), a.size, _kt(a)))


def mono(a: np.ndarray) -> int:
    """Mono(A): fewest monotone (sorted or reversely sorted) pieces."""
    a = np.ascontiguousarray(a)
    return int(_load().sro_mono(_ptr(a), a.size, _kt(a)))


def inversions(a: np.ndarray) -> int:
    """Inv(A) by its O(n^2) definition."""
    a = np.ascontiguousarray(a)
    return int(_load().sro_inversions(_ptr(a), a.size, _kt(a)))


def rem(a: np.ndarray) -> int:
    """Rem(A): fewest items whose removal leaves a sorted list."""
    a = np.ascontiguousarray(a)
    return int(_load().sro_rem(_ptr(a), a.size, _kt(a)))


def comparisons() -> int:
    return int(_load().sro_cmp_count())


def reset_comparisons() -> None:
    _load().sro_cmp_reset()


TRACE_EVENTS = {1: "trim_a", 2: "trim_b", 3: "copy_a", 4: "copy_b", 5: "gallop_a", 6: "gallop_b"}


def sort_with_trace(keys: np.ndarray):
    """Mergesorts a copy of ``keys`` with the paper's mer5 (natural runs, no
    growth of short runs, so the runs merged are the input's own, as in the
    worked example of Section 3) and returns (sorted, [(event, count), ...])
    listing what every merge did."""
    lib = _load()
    lib.sro_trace_enable(1)
    try:
        out = sort_keys(keys, "merge5")
        buf = np.zeros(256, dtype=np.int64)
        k = lib.sro_trace_read(_ptr(buf), 256)
    finally:
        lib.sro_trace_enable(0)
    ev = [(TRACE_EVENTS[int(buf[i])], int(buf[i + 1])) for i in range(0, k, 2)]
    return out, ev
