"""Thin Python binding of libsortrace_gb300.so (the C ABI in include/sortrace.h).

Only argument marshalling happens here: device pointers and the current CUDA
stream are taken from PyTorch tensors and passed to the C entry points, which
run every step of the sort in the library's own CUDA kernels.  There is no CPU
path: if the library is missing the calls raise.

    import paper_1609_04471_gb300 as sr
    sr.sort_keys(x)                   # x: CUDA tensor, sorted in place
    sr.sort_pairs(keys, vals)         # stable, in place
    sr.sort_segmented(keys, offsets)  # every segment on its own
    sr.sort_keys_learned(x)           # learned partition, same output as sort_keys
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsortrace_gb300.so")

KEY_I32, KEY_U32, KEY_F32, KEY_U64, KEY_I64 = 0, 1, 2, 3, 4
STATUS = {0: "SR_OK", 1: "SR_ERR_INVALID_ARG", 2: "SR_ERR_UNSUPPORTED", 3: "SR_ERR_OOM",
          4: "SR_ERR_CUDA", 5: "SR_ERR_TIMEOUT", 6: "SR_ERR_INTERNAL", 7: "SR_ERR_BAD_SEGMENTS"}
MODEL_TRAINED, MODEL_EQUAL_WIDTH, MODEL_UNTRAINED, MODEL_FORCE_BAD = 0, 1, 2, 3
MODEL_HIDDEN, MODEL_PARAMS = 32, 65

_lock = threading.Lock()
_lib = None


class SortError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class RunInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("runs", ctypes.c_uint64), ("sorted", ctypes.c_int32),
                ("strictly_descending", ctypes.c_int32), ("tile", ctypes.c_uint64),
                ("tiles", ctypes.c_uint64), ("tiles_ascending", ctypes.c_uint64),
                ("tiles_descending", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("abi_version", ctypes.c_uint32), ("call", ctypes.c_int32), ("n", ctypes.c_uint64),
                ("key_type", ctypes.c_int32), ("tile", ctypes.c_int32), ("merge_tile", ctypes.c_int32),
                ("passes_planned", ctypes.c_int32), ("passes_skipped", ctypes.c_int32),
                ("input_class", ctypes.c_int32), ("fallback", ctypes.c_int32),
                ("runs", ctypes.c_uint64), ("bytes_moved", ctypes.c_uint64),
                ("max_bucket", ctypes.c_uint64), ("big_segments", ctypes.c_uint64),
                ("model_loss", ctypes.c_float), ("bucket_imbalance", ctypes.c_float),
                ("displaced", ctypes.c_uint64)]


class LearnedOpts(ctypes.Structure):
    _fields_ = [("num_buckets", ctypes.c_uint32), ("sample_stride", ctypes.c_uint32),
                ("train_points", ctypes.c_uint32), ("train_steps", ctypes.c_uint32),
                ("learning_rate", ctypes.c_float), ("model", ctypes.c_uint32),
                ("bucket_config", ctypes.c_uint32)]


# name -> (restype, argtypes) of every entry point declared in include/sortrace.h
_vp, _sz, _i32, _u32, _u64, _fp = (ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                   ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p)
SIGNATURES = {
    "sr_sort_keys": (_i32, [_vp, _sz, _i32, _vp]),
    "sr_sort_pairs": (_i32, [_vp, _vp, _sz, _i32, _vp]),
    "sr_sort_segmented": (_i32, [_vp, _vp, _sz, _i32, _vp]),
    "sr_sort_segmented_ex": (_i32, [_vp, _sz, _vp, _sz, _i32, _vp]),
    "sr_sort_segmented_cfg": (_i32, [_vp, _sz, _vp, _sz, _i32, _i32, _vp]),
    "sr_segmented_num_configs": (_i32, [_i32]),
    "sr_segmented_config_info": (_i32, [_i32, _i32, _vp]),
    "sr_sort_keys_host": (_i32, [_vp, _sz, _i32, _vp]),
    "sr_sort_keys_host_async": (_i32, [_vp, _sz, _i32, _vp]),
    "sr_sort_keys_host_many": (_i32, [_vp, _vp, _i32, _i32, _vp]),
    "sr_release_cached": (_i32, []),
    "sr_sort_keys_noalloc": (_i32, [_vp, _sz, _i32, _vp]),
    "sr_sort_keys_learned": (_i32, [_vp, _sz, _i32, _vp, _vp]),
    "sr_detect_runs": (_i32, [_vp, _sz, _i32, _vp, _vp]),
    "sr_get_stats": (_i32, [_vp]),
    "sr_stream_status": (_i32, [_vp]),
    "sr_status_string": (ctypes.c_char_p, [_i32]),
    "sr_model_loss_grad": (_i32, [_vp, _vp, _sz, _vp, _vp, _vp, _vp]),
    "sr_model_train": (_i32, [_vp, _vp, _sz, _vp, _u32, ctypes.c_float, _vp, _vp]),
    "sr_model_buckets": (_i32, [_vp, _sz, _i32, _vp, _u64, _u64, _u32, _vp, _vp]),
    "sr_launch_count": (_u64, []),
    "sr_profile_begin": (_i32, []),
    "sr_profile_end": (_i32, [_vp, _i32]),
}

KERNEL_KINDS = ("detect", "reverse", "block_sort", "partition", "merge", "copy", "segmented", "model", "displaced")


class SegmentedConfig(ctypes.Structure):
    _fields_ = [("strategy", ctypes.c_int32), ("sort_threads", ctypes.c_int32),
                ("pack_items", ctypes.c_int32), ("tile_items", ctypes.c_int32),
                ("fan_in", ctypes.c_int32), ("merge_threads", ctypes.c_int32),
                ("tile_keys", ctypes.c_int64), ("cta_keys", ctypes.c_int64),
                ("small_keys", ctypes.c_int64), ("ladder", ctypes.c_int32), ("reserved", ctypes.c_int32)]


SEG_CONFIG_DEFAULT = -1


class KernelTime(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("ms", ctypes.c_double)]


def load(path: str | None = None):
    """Loads the library (building it first if it is absent and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            from . import _build
            _build.build()
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(code: int, what: str) -> None:
    if code != 0:
        raise SortError(code, what)


def key_type_of(t) -> int:
    import torch
    m = {torch.int32: KEY_I32, torch.float32: KEY_F32, torch.int64: KEY_I64}
    for name, kt in (("uint32", KEY_U32), ("uint64", KEY_U64)):
        dt = getattr(torch, name, None)
        if dt is not None:
            m[dt] = kt
    try:
        return m[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported key dtype {t.dtype}") from None


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _cuda_contig(t, what):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")


def sort_keys(x, key_type: int | None = None, stream=None):
    """Sorts the CUDA tensor x in place (ascending); returns x."""
    _cuda_contig(x, "keys")
    kt = key_type_of(x) if key_type is None else key_type
    _check(load().sr_sort_keys(x.data_ptr(), x.numel(), kt, _stream(stream)), "sr_sort_keys")
    return x


NOALLOC_MAX_KEYS = 1 << 20


def sort_keys_noalloc(x, key_type: int | None = None, stream=None):
    """sort_keys without any device allocation (at most NOALLOC_MAX_KEYS keys;
    calls must not overlap on the device)."""
    _cuda_contig(x, "keys")
    kt = key_type_of(x) if key_type is None else key_type
    _check(load().sr_sort_keys_noalloc(x.data_ptr(), x.numel(), kt, _stream(stream)),
           "sr_sort_keys_noalloc")
    return x


def sort_pairs(keys, vals, key_type: int | None = None, stream=None):
    """Stable sort of (keys, vals) by key, in place; vals is int32/uint32."""
    _cuda_contig(keys, "keys")
    _cuda_contig(vals, "vals")
    if vals.element_size() != 4 or vals.numel() != keys.numel():
        raise ValueError("vals must hold one 4-byte payload per key")
    kt = key_type_of(keys) if key_type is None else key_type
    _check(load().sr_sort_pairs(keys.data_ptr(), vals.data_ptr(), keys.numel(), kt, _stream(stream)),
           "sr_sort_pairs")
    return keys, vals


def sort_segmented(keys, offsets, key_type: int | None = None, stream=None):
    """Sorts every segment keys[offsets[s]:offsets[s+1]] in place; offsets is
    an int64 CUDA tensor of num_segments + 1 entries."""
    _cuda_contig(keys, "keys")
    _cuda_contig(offsets, "offsets")
    import torch
    if offsets.dtype != torch.int64:
        raise ValueError("offsets must be int64")
    kt = key_type_of(keys) if key_type is None else key_type
    _check(load().sr_sort_segmented(keys.data_ptr(), offsets.data_ptr(), max(offsets.numel() - 1, 0),
                                    kt, _stream(stream)), "sr_sort_segmented")
    return keys


def sort_segmented_ex(keys, offsets, key_type: int | None = None, stream=None):
    """sort_segmented without reading the total length back (graph-capturable)."""
    _cuda_contig(keys, "keys")
    _cuda_contig(offsets, "offsets")
    kt = key_type_of(keys) if key_type is None else key_type
    _check(load().sr_sort_segmented_ex(keys.data_ptr(), keys.numel(), offsets.data_ptr(),
                                       max(offsets.numel() - 1, 0), kt, _stream(stream)),
           "sr_sort_segmented_ex")
    return keys


def sort_segmented_cfg(keys, offsets, config: int, key_type: int | None = None, stream=None):
    """sort_segmented_ex under launch configuration `config` (an index of
    segmented_configs(key_type), or SEG_CONFIG_DEFAULT)."""
    _cuda_contig(keys, "keys")
    _cuda_contig(offsets, "offsets")
    kt = key_type_of(keys) if key_type is None else key_type
    _check(load().sr_sort_segmented_cfg(keys.data_ptr(), keys.numel(), offsets.data_ptr(),
                                        max(offsets.numel() - 1, 0), kt, int(config), _stream(stream)),
           "sr_sort_segmented_cfg")
    return keys


def segmented_configs(key_type: int) -> list:
    """The segmented sort's launch configurations for a key type, as dicts."""
    lib = load()
    out = []
    for i in range(lib.sr_segmented_num_configs(key_type)):
        c = SegmentedConfig()
        _check(lib.sr_segmented_config_info(key_type, i, ctypes.byref(c)), "sr_segmented_config_info")
        d = {f: getattr(c, f) for f, _ in SegmentedConfig._fields_}
        d["index"] = i
        out.append(d)
    return out


def sort_keys_learned(x, key_type: int | None = None, stream=None, **opts):
    """Learned-partition sort of the CUDA tensor x in place; same output as
    sort_keys.  opts: num_buckets, sample_stride, train_points, train_steps,
    learning_rate, model, bucket_config (1 + a segmented configuration
    index; 0 for the default)."""
    _cuda_contig(x, "keys")
    kt = key_type_of(x) if key_type is None else key_type
    o = LearnedOpts()
    for k, v in opts.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    _check(load().sr_sort_keys_learned(x.data_ptr(), x.numel(), kt, ctypes.byref(o), _stream(stream)),
           "sr_sort_keys_learned")
    return x


def _host_args(arr, key_type):
    import numpy as np
    if isinstance(arr, np.ndarray):
        if not arr.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        kt = key_type if key_type is not None else {
            np.dtype(np.int32): KEY_I32, np.dtype(np.uint32): KEY_U32, np.dtype(np.float32): KEY_F32,
            np.dtype(np.uint64): KEY_U64, np.dtype(np.int64): KEY_I64}[arr.dtype]
        ptr, n = arr.ctypes.data, arr.size
    else:
        if arr.is_cuda or not arr.is_contiguous():
            raise ValueError("host tensor must be a contiguous CPU tensor")
        kt = key_type_of(arr) if key_type is None else key_type
        ptr, n = arr.data_ptr(), arr.numel()
    return ptr, n, kt


def sort_keys_host(arr, key_type: int | None = None, stream=None):
    """Sorts a host (CPU) tensor or numpy array in place through the device:
    copy in, sort, copy out, wait."""
    ptr, n, kt = _host_args(arr, key_type)
    _check(load().sr_sort_keys_host(ptr, n, kt, _stream(stream)), "sr_sort_keys_host")
    return arr


def sort_keys_host_async(arr, key_type: int | None = None, stream=None):
    """sort_keys_host queued on the stream without waiting; `arr` must be in
    page-locked memory (e.g. torch's pin_memory()) and left alone until the
    stream completes."""
    ptr, n, kt = _host_args(arr, key_type)
    _check(load().sr_sort_keys_host_async(ptr, n, kt, _stream(stream)), "sr_sort_keys_host_async")
    return arr


def sort_keys_host_many(arrs, key_type: int | None = None, stream=None):
    """Sorts several page-locked host arrays in place as a pipeline (copy in,
    sort, copy out overlap across arrays), queued on the stream without
    waiting; the arrays must be left alone until the stream completes."""
    args = [_host_args(a, key_type) for a in arrs]
    kts = {kt for _, _, kt in args}
    if len(kts) > 1:
        raise ValueError("all arrays must have one key type")
    ptrs = (ctypes.c_void_p * len(args))(*[p for p, _, _ in args])
    ns = (ctypes.c_size_t * len(args))(*[n for _, n, _ in args])
    kt = kts.pop() if kts else (key_type if key_type is not None else KEY_I32)
    _check(load().sr_sort_keys_host_many(ptrs, ns, len(args), kt, _stream(stream)), "sr_sort_keys_host_many")
    return arrs


def release_cached():
    """Drops the graphs kept for repeated sort calls on the current device
    (and their scratch); later calls build them again."""
    _check(load().sr_release_cached(), "sr_release_cached")


def detect_runs(x, key_type: int | None = None, stream=None) -> dict:
    """Runs the run-detection scan on x and returns its counts."""
    _cuda_contig(x, "keys")
    kt = key_type_of(x) if key_type is None else key_type
    info = RunInfo()
    _check(load().sr_detect_runs(x.data_ptr(), x.numel(), kt, ctypes.byref(info), _stream(stream)),
           "sr_detect_runs")
    return {f: getattr(info, f) for f, _ in RunInfo._fields_}


def stats() -> dict:
    """Statistics of this thread's last sort call (waits for its stream)."""
    st = Stats()
    _check(load().sr_get_stats(ctypes.byref(st)), "sr_get_stats")
    return {f: getattr(st, f) for f, _ in Stats._fields_}


def stream_status(stream=None) -> int:
    """Waits for the stream and returns (and clears) the device status word."""
    return int(load().sr_stream_status(_stream(stream)))


def launch_count() -> int:
    """Number of kernels the library has launched in this process."""
    return int(load().sr_launch_count())


def profile_begin() -> None:
    """Brackets every following launch of this thread with CUDA events."""
    _check(load().sr_profile_begin(), "sr_profile_begin")


def profile_end() -> dict:
    """Waits for the bracketed launches; returns {kind: (launches, ms)}."""
    arr = (KernelTime * len(KERNEL_KINDS))()
    _check(load().sr_profile_end(arr, len(KERNEL_KINDS)), "sr_profile_end")
    return {k: (int(arr[i].launches), float(arr[i].ms)) for i, k in enumerate(KERNEL_KINDS)}


def model_loss_grad(x, t, theta, stream=None):
    """Loss and gradient of the router network on the device: x, t float32
    CUDA tensors; theta a sequence of 65 floats.  Returns (loss, grad list)."""
    _cuda_contig(x, "x")
    _cuda_contig(t, "t")
    th = (ctypes.c_float * MODEL_PARAMS)(*[float(v) for v in theta])
    g = (ctypes.c_float * MODEL_PARAMS)()
    loss = ctypes.c_float()
    _check(load().sr_model_loss_grad(x.data_ptr(), t.data_ptr(), x.numel(), th, ctypes.byref(loss), g,
                                     _stream(stream)), "sr_model_loss_grad")
    return float(loss.value), list(g)


def model_train(x, t, theta, steps: int, lr: float, stream=None):
    """Adam steps on the device; returns (theta list, final loss)."""
    _cuda_contig(x, "x")
    _cuda_contig(t, "t")
    th = (ctypes.c_float * MODEL_PARAMS)(*[float(v) for v in theta])
    loss = ctypes.c_float()
    _check(load().sr_model_train(x.data_ptr(), t.data_ptr(), x.numel(), th, steps, lr, ctypes.byref(loss),
                                 _stream(stream)), "sr_model_train")
    return list(th), float(loss.value)


def model_buckets(keys, theta, lo: int, hi: int, num_buckets: int, out, key_type: int | None = None,
                  stream=None):
    """Bucket of every key under the router network, into out (uint32/int32)."""
    _cuda_contig(keys, "keys")
    _cuda_contig(out, "out")
    kt = key_type_of(keys) if key_type is None else key_type
    th = (ctypes.c_float * MODEL_PARAMS)(*[float(v) for v in theta])
    _check(load().sr_model_buckets(keys.data_ptr(), keys.numel(), kt, th, lo, hi, num_buckets,
                                   out.data_ptr(), _stream(stream)), "sr_model_buckets")
    return out
