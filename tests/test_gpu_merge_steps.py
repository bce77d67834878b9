"""GPU parity of the merge steps against the CPU oracle, bit for bit, through
the C ABI: the 4-way steps (the default for payloads and 8-byte keys) and the
2-way steps (the default for 4-byte keys), each with its three ways of staging
a tile (1-D bulk copies for 16-byte aligned arrays, 16-byte loads through
registers, scalar loads for unaligned arrays), at sizes around every tile and
group boundary and with ragged tails.  The staging and fan-in switches are
read once per process, so the forced runs go through child processes."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import sortrace_inputs as si

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KT = {np.dtype(np.int32): 0, np.dtype(np.uint32): 1, np.dtype(np.float32): 2,
      np.dtype(np.uint64): 3, np.dtype(np.int64): 4}


def _random(rng, n, dtype, alphabet=None):
    if alphabet:
        return rng.integers(0, alphabet, n).astype(dtype)
    if dtype == np.float32:
        b = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        b[np.isnan(b.view(np.float32))] = 0x3F800000
        return b.view(np.float32)
    if dtype in (np.uint64, np.int64):
        return rng.integers(0, 1 << 64, n, dtype=np.uint64).view(dtype)
    return rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32).view(dtype)


def _sizes(sr, kb, vals=False):
    """Sizes around the merge tile (nv), the block-sort tile (ts) and 4-way
    groups of 1, 2, 4 and 16 tiles, with ragged tails."""
    import torch
    t = torch.zeros(1000, dtype={4: torch.int32, 8: torch.int64}[kb], device="cuda")
    if vals:
        sr.sort_pairs(t, torch.zeros(1000, dtype=torch.int32, device="cuda"), key_type=0 if kb == 4 else 3)
    else:
        sr.sort_keys(t, key_type=0 if kb == 4 else 3)
    st = sr.stats()
    nv, ts = st["merge_tile"], st["tile"]
    out = {nv + 1, ts + 1, 2 * ts - 1, 2 * ts + 3, 3 * ts + 5, 4 * ts, 4 * ts + 1, 5 * ts + 7, 8 * ts + 2,
           16 * ts - 3, 16 * ts + nv + 1, 17 * ts + 1, 64 * ts + 3, 65 * ts + 1}
    return sorted(out)


def _tile(sr):
    """The block-sort tile of 4-byte keys alone, as the library's statistics
    report it after a small sort."""
    import torch
    sr.sort_keys(torch.zeros(1000, dtype=torch.int32, device="cuda"), key_type=0)
    return sr.stats()["tile"]


def _dev(a, offset=0):
    """A device copy of a; offset > 0 puts it that many elements past a
    16-byte boundary (a view into a larger buffer)."""
    import torch
    bits = {4: torch.int32, 8: torch.int64}[a.dtype.itemsize]
    buf = torch.zeros(a.size + offset, dtype=bits, device="cuda")
    buf[offset:] = torch.from_numpy(np.ascontiguousarray(a).view({4: np.int32, 8: np.int64}[a.dtype.itemsize])).cuda()
    return buf, buf[offset:]


@pytest.mark.parametrize("dtype", [np.int32, np.float32, np.uint64, np.int64])
@pytest.mark.parametrize("offset", [0, 1])
def test_keys_steps(gpu_lib, dtype, offset):
    """Keys at every boundary size, random and few-valued, aligned (bulk
    copies) and one element off (scalar staging)."""
    rng = np.random.default_rng(70 + offset)
    for n in _sizes(gpu_lib, np.dtype(dtype).itemsize):
        for alphabet in (None, 5):
            a = _random(rng, n, dtype, alphabet)
            buf, x = _dev(a, offset)
            gpu_lib.sort_keys(x, key_type=KT[np.dtype(dtype)])
            got = x.cpu().numpy().view(dtype)
            assert got.tobytes() == oracle.sort_keys(a).tobytes(), (dtype, n, offset, alphabet)
            if offset:
                assert int(buf[0]) == 0
    assert gpu_lib.stream_status() == 0


@pytest.mark.parametrize("dtype", [np.int32, np.uint64])
@pytest.mark.parametrize("offset", [0, 1])
def test_pairs_steps(gpu_lib, dtype, offset):
    """Stable pairs at every boundary size with many equal keys: payloads of
    equal keys keep their input order through the 4-way steps."""
    import torch
    rng = np.random.default_rng(80 + offset)
    for n in _sizes(gpu_lib, np.dtype(dtype).itemsize, vals=True):
        k = _random(rng, n, dtype, alphabet=7 if n % 2 else None)
        v = np.arange(n, dtype=np.uint32)
        _, xk = _dev(k, offset)
        vbuf = torch.zeros(n + offset, dtype=torch.int32, device="cuda")
        vbuf[offset:] = torch.from_numpy(v.view(np.int32)).cuda()
        gpu_lib.sort_pairs(xk, vbuf[offset:], key_type=KT[np.dtype(dtype)])
        ok, ov = oracle.sort_pairs(k, v)
        assert xk.cpu().numpy().view(dtype).tobytes() == ok.tobytes(), (dtype, n, offset)
        assert vbuf[offset:].cpu().numpy().view(np.uint32).tobytes() == ov.tobytes(), (dtype, n, offset)
    assert gpu_lib.stream_status() == 0


def test_presorted_groups_skip_steps(gpu_lib):
    """Tiles whose runs are already in order at the 4-way levels: those steps
    are skipped (statistics) and the result still equals the oracle's."""
    import torch
    st0 = None
    ts = _tile(gpu_lib)
    for n in (64 * ts + 5, 33 * ts):
        a = np.sort(si.uniform_i32(n, 5))
        # shuffle inside each block-sort tile only: every merge level is in order
        rng = np.random.default_rng(5)
        for t0 in range(0, n, ts):
            seg = a[t0:t0 + ts].copy()
            rng.shuffle(seg)
            a[t0:t0 + ts] = seg
        x = torch.from_numpy(a.copy()).cuda()
        gpu_lib.sort_keys(x, key_type=0)
        st0 = gpu_lib.stats()
        assert x.cpu().numpy().tobytes() == oracle.sort_keys(a).tobytes()
        assert st0["passes_skipped"] == st0["passes_planned"] > 0


_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import paper_1609_04471_gb300 as sr, oracle, sortrace_inputs as si
rng = np.random.default_rng(9)
sr.sort_keys(torch.zeros(1000, dtype=torch.int32, device="cuda"), key_type=0)
ts = sr.stats()["tile"]
sizes = [ts + 1, 2 * ts + 3, 4 * ts + 1, 5 * ts + 7, 17 * ts + 1, (1 << 20) + 3]
for n in sizes:
    for dt, kt in ((np.int32, 0), (np.uint64, 3)):
        a = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(dt) if dt == np.int32 else \
            rng.integers(0, 1 << 64, n, dtype=np.uint64)
        x = torch.from_numpy(a.view(np.int32 if dt == np.int32 else np.int64).copy()).cuda()
        sr.sort_keys(x, key_type=kt)
        assert x.cpu().numpy().view(dt).tobytes() == oracle.sort_keys(a).tobytes(), (n, dt)
    k = rng.integers(0, 9, n).astype(np.int32)
    v = np.arange(n, dtype=np.uint32)
    xk = torch.from_numpy(k.copy()).cuda()
    xv = torch.from_numpy(v.view(np.int32).copy()).cuda()
    sr.sort_pairs(xk, xv, key_type=0)
    ok, ov = oracle.sort_pairs(k, v)
    assert xk.cpu().numpy().tobytes() == ok.tobytes() and xv.cpu().numpy().view(np.uint32).tobytes() == ov.tobytes()
assert sr.stream_status() == 0
a = si.uniform_i32(1 << 24, 3)
x = torch.from_numpy(a.copy()).cuda()
sr.sort_keys(x, key_type=0)
assert x.cpu().numpy().tobytes() == oracle.sort_keys(a).tobytes()
print("child ok", sr.stats()["passes_planned"], ts)
"""


@pytest.mark.parametrize("env", [{"SORTRACE_MERGE_FANIN": "4"},
                                 {"SORTRACE_MERGE_FANIN": "4", "SORTRACE_MERGE4_STAGE": "vec"},
                                 {"SORTRACE_MERGE_FANIN": "2"},
                                 {"SORTRACE_MERGE_FANIN": "2", "SORTRACE_MERGE2_STAGE": "vec"}])
def test_other_staging_and_fanin(env):
    """Every key shape forced to 4-way steps (bulk-copy staging, then 16-byte
    register staging), and to 2-way steps (bulk copies, then 16-byte register
    staging), in child processes: the same sizes and classes against the
    oracle."""
    e = dict(os.environ)
    e.update(env)
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], env=e, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "child ok" in r.stdout
    planned, ts = (int(x) for x in r.stdout.split("child ok")[1].split()[:2])
    levels = int(np.ceil(np.log2(-(-(1 << 24) // ts))))     # binary merge levels over 2^24 int32 keys
    assert planned == ((levels + 1) // 2 if env.get("SORTRACE_MERGE_FANIN") == "4" else levels)


def test_descending_tile_chains(gpu_lib):
    """Inputs whose block-sorted tiles come in descending order (k-even and
    k-sharp teeth, non-increasing lists with long blocks of equal keys that
    straddle tile boundaries): the block sort writes such chains reversed, the
    merge steps finish; keys and stable pairs equal the oracle's at sizes
    where the block sort writes to the other buffer and where it works in
    place."""
    import torch
    ts = _tile(gpu_lib)
    for n in (64 * ts, 64 * ts + 77, 32 * ts + 5, 33 * ts):
        rng = np.random.default_rng(n)
        cases = [si.k_even_teeth(n - n % 4, 4), si.k_sharp_teeth(n - n % 8, 8),
                 np.repeat(np.arange(n // 5000 + 1, dtype=np.int32)[::-1], 5000)[:n],
                 np.sort(rng.integers(0, 50, n).astype(np.int32))[::-1].copy()]
        for a in cases:
            x = torch.from_numpy(a.copy()).cuda()
            gpu_lib.sort_keys(x, key_type=0)
            assert x.cpu().numpy().tobytes() == oracle.sort_keys(a).tobytes(), n
            v = np.arange(a.size, dtype=np.uint32)
            xk = torch.from_numpy(a.copy()).cuda()
            xv = torch.from_numpy(v.view(np.int32).copy()).cuda()
            gpu_lib.sort_pairs(xk, xv, key_type=0)
            ok, ov = oracle.sort_pairs(a, v)
            assert xk.cpu().numpy().tobytes() == ok.tobytes(), n
            assert xv.cpu().numpy().view(np.uint32).tobytes() == ov.tobytes(), n
            u = a.astype(np.int64) * 3 - 7
            x8 = torch.from_numpy(u.copy()).cuda()
            gpu_lib.sort_keys(x8, key_type=4)
            assert x8.cpu().numpy().tobytes() == oracle.sort_keys(u).tobytes(), n
    assert gpu_lib.stream_status() == 0
