"""The C ABI without a GPU: the library builds for sm_103a, loads, exports
every entry point include/sortrace.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sr_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1609_04471_gb300 import _build
    import paper_1609_04471_gb300 as sr
    _build.build()
    return sr.load()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("sr_sort_keys", "sr_sort_pairs", "sr_sort_segmented", "sr_sort_keys_learned",
                 "sr_get_stats", "sr_stream_status", "sr_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_1609_04471_gb300 as sr
    assert set(sr.SIGNATURES) == _declared()


def test_status_strings(lib):
    assert lib.sr_status_string(0) == b"SR_OK"
    assert lib.sr_status_string(7) == b"SR_ERR_BAD_SEGMENTS"
    assert lib.sr_status_string(99) == b"SR_ERR_UNKNOWN"


def test_argument_errors_need_no_device(lib):
    # unknown key type, null pointers with n > 1, misaligned pointers: rejected
    # before any CUDA call; n <= 1 is a no-op
    assert lib.sr_sort_keys(None, 10, 9, None) == 1
    assert lib.sr_sort_keys(None, 10, 0, None) == 1
    assert lib.sr_sort_keys(ctypes.c_void_p(2), 10, 0, None) == 1
    assert lib.sr_sort_keys(None, 1, 0, None) == 0
    assert lib.sr_sort_keys(None, 0, 3, None) == 0
    assert lib.sr_sort_pairs(ctypes.c_void_p(256), None, 5, 0, None) == 1
    assert lib.sr_sort_pairs(None, None, 1, 0, None) == 0
    assert lib.sr_detect_runs(None, 4, 0, None, None) == 1
    assert lib.sr_get_stats(None) == 1
    # several host arrays: a bad key type, a negative count, missing arrays
    n = (ctypes.c_size_t * 1)(10)
    assert lib.sr_sort_keys_host_many(None, n, 1, 9, None) == 1
    assert lib.sr_sort_keys_host_many(None, None, -1, 0, None) == 1
    assert lib.sr_sort_keys_host_many(None, n, 1, 0, None) == 1


def test_segmented_configs_described_without_gpu():
    """The configuration table is host data: every entry is consistent and an
    unknown entry is refused before anything reaches the GPU."""
    import ctypes
    import paper_1609_04471_gb300 as sr
    lib = sr.load()
    for kt in range(5):
        n = lib.sr_segmented_num_configs(kt)
        assert n >= 3
        for i in range(n):
            c = sr.SegmentedConfig()
            assert lib.sr_segmented_config_info(kt, i, ctypes.byref(c)) == 0
            assert c.tile_keys == c.sort_threads * c.tile_items
            assert c.cta_keys == c.fan_in * c.tile_keys
            assert c.fan_in in (1, 2, 4) and c.tile_items % 2 == 1
            assert c.strategy in (0, 1) and (c.pack_items > 0) == (c.strategy == 0)
            assert 0 < c.small_keys <= c.cta_keys
        c = sr.SegmentedConfig()
        assert lib.sr_segmented_config_info(kt, n, ctypes.byref(c)) == 1
        assert lib.sr_segmented_config_info(kt, -1, ctypes.byref(c)) == 0     # the default
        assert lib.sr_sort_segmented_cfg(None, 0, None, 0, kt, n, None) == 1
    assert lib.sr_segmented_num_configs(9) == 0
