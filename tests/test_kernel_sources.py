"""Static checks on the CUDA sources.

Every kernel is launched with programmatic dependent launch, so its CTAs may
start while the previous kernel on the stream is still running; each kernel
must therefore call griddep_wait() before it reads anything.  No kernel may
trap or assert on the device."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1609_04471_gb300", "csrc")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")))


def _kernel_bodies(src):
    for m in re.finditer(r"__global__\s+void[^;{]*?\b(k_\w+)\s*\([^{;]*\)\s*\{", src, re.S):
        yield m.group(1), src[m.end():m.end() + 400]


def test_every_kernel_waits_for_its_predecessor():
    seen = 0
    for path in _sources():
        src = open(path).read()
        for name, body in _kernel_bodies(src):
            seen += 1
            first = body.strip().split(";")[0].strip()
            assert first == "griddep_wait()", f"{os.path.basename(path)}:{name} starts with {first!r}"
    assert seen >= 7


def test_no_device_traps():
    for path in _sources():
        src = open(path).read()
        assert "__trap" not in src and "trap;" not in src, path
        assert not re.search(r"\bassert\s*\(", src), path
