"""Host-side units of the library built and run on the CPU: the split of a
bitsliced launch's (block, tile) work items into per-CTA ranges, checked on
20 000 random shapes (endpoints, order, and every CTA within one tile's cost
of an equal share)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1412_3022_gb300", "csrc")


def test_bitsliced_cta_ranges():
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not found")
    out_dir = os.path.join(ROOT, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "test_cta_ranges")
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-I" + CSRC, "-o", exe,
                        os.path.join(ROOT, "tests", "host", "cta_ranges.cpp"),
                        os.path.join(CSRC, "bs_emit.cpp")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
