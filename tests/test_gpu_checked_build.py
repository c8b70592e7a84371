"""The checked build (compiled with IFDK_CHECK): every tap read of the packed
back-projector is tested against its stage's TMA box, and a read outside it
would set the plan's status to IFDK_ERR_BOUNDS (the read itself is redirected
inside the box).  The packed, random-geometry, degenerate-shape, streaming,
shard (pair ranges: blocks that start at any pair), batch and quad suites run
against that library in a subprocess.  They assert a clean device
status after their launches, and parity with the oracle as usual."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_keeps_every_tap_read_in_its_window():
    pytest.importorskip("torch")
    from paper_1909_02724_gb300.build import build_checked
    lib = build_checked()
    env = dict(os.environ, IFDK_LIB_PATH=lib)
    suites = ["tests/test_gpu_packed.py", "tests/test_gpu_random_geometries.py", "tests/test_gpu_degenerate.py",
              "tests/test_gpu_stream.py", "tests/test_gpu_shards.py", "tests/test_gpu_batches.py",
              "tests/test_gpu_quads.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", *suites],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
