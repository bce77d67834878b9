import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library, built in-tree; a missing extension is an error, never
    a fallback."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    import paper_1609_04471_gb300 as sr
    sr.load()
    return sr


def _sha256(*arrays):
    import hashlib

    import numpy as np
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).view(np.uint8).data)
    return h.hexdigest()


@pytest.fixture(scope="session")
def full_size_oracle():
    """check(name, inputs, outputs, run_oracle): compares every byte of a
    full-size GPU result with the oracle's.  The oracle's digest for the
    seeded input is read from tests/golden/full_size_digests.json (written by
    tests/golden/make_full_size_digests.py, which calls only the oracle and
    the input generators); if this machine generated a different input, the
    oracle runs here instead and its output is compared in full."""
    import json

    import numpy as np
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size_digests.json")
    with open(path) as f:
        golden = json.load(f)

    def check(name, inputs, outputs, run_oracle):
        g = golden[name]
        if _sha256(*inputs) == g["input_sha256"]:
            assert _sha256(*outputs) == g["oracle_output_sha256"], f"{name}: GPU output differs from the oracle's"
            return "digest"
        want = run_oracle()
        for got, w in zip(outputs, want):
            assert np.ascontiguousarray(got).tobytes() == np.ascontiguousarray(w).tobytes(), name
        return "oracle"

    return check
