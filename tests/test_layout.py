"""The workspace layout, checked on the host (no GPU): tests/layout_check.cu
is compiled with nvcc as host code and asserts that every region is
256-byte aligned and disjoint from the next, that the per-call zeroed range
holds the control records the kernels expect to be zero and not the
self-resetting slots, for single sets and batches of several sizes."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc (host compilation only)")
def test_layout_regions(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "layout_check")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-x", "cu",
                    os.path.join(HERE, "layout_check.cu"), "-o", exe], check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
    assert "layout ok" in r.stdout
