"""Writes full_size_digests.json: for each full-size workload, the SHA-256 of
its seeded input and of the CPU oracle's sorted output.

The GPU parity tests at full size (2^28 int32 keys, 2^28 uint64 + uint32
stable pairs, 2^27 float32 keys for the learned sort, the 200,000-array batch)
hash every byte of the GPU's output and compare it with the oracle's digest
recorded here; a digest equal for all bytes is an element-by-element
comparison.  If the input generated on the test machine hashes differently
(another libm could round a float draw differently), the tests run the oracle
there instead.

This script calls only the oracle and the seeded input generators; nothing
in it comes from the GPU library.  Run from the repository root:

    python tests/golden/make_full_size_digests.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import sortrace_inputs as si  # noqa: E402

OUT = os.path.join(HERE, "full_size_digests.json")


def sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).view(np.uint8).data)
    return h.hexdigest()


def uniform_2_28():
    a = si.uniform_i32(1 << 28, 1)
    return sha(a), sha(oracle.sort_keys(a))


def pairs_2_28():
    k, v = si.pairs_u64_zipf(1 << 28, 1)
    d_in = sha(k, v)
    ok, ov = oracle.sort_pairs(k, v)
    return d_in, sha(ok, ov)


def lognormal_2_27():
    a = si.lognormal_f32(1 << 27, 1)
    return sha(a), sha(oracle.sort_keys(a))


def batch_200k():
    keys, off, _ = si.segmented_i32(200_000, 1)
    return sha(keys, off), sha(oracle.sort_segmented(keys, off))


CASES = {
    "uniform_i32_2p28_seed1": ("2^28 int32 keys, uniform over the full range, seed 1", uniform_2_28),
    "pairs_u64_zipf_2p28_seed1": ("2^28 stable pairs: uint64 keys (half uniform, half Zipf s=1.1 over "
                                  "2^20 values), uint32 payload = index, seed 1", pairs_2_28),
    "lognormal_f32_2p27_seed1": ("2^27 float32 keys from the lognormal mixture, seed 1", lognormal_2_27),
    "batch_200k_seed1": ("200,000 int32 arrays, lognormal lengths (median 512), four classes, seed 1",
                         batch_200k),
}


def main(names=None):
    res = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            res = json.load(f)
    for name, (what, fn) in CASES.items():
        if names and name not in names:
            continue
        t = time.time()
        d_in, d_out = fn()
        res[name] = {"what": what, "input_sha256": d_in, "oracle_output_sha256": d_out}
        print(f"{name}: {time.time() - t:.1f} s", flush=True)
        with open(OUT, "w") as f:
            json.dump(res, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or None)
