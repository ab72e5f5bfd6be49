"""The library's layout arithmetic, compiled from its own header and run on
the host: the vEB slot function against the paper's worked example and as a
bijection, the segments of a level (left child ceil(m/2), reading G3), the
tree height, and the packed k-NN record numbering (every record once,
entries that are records or leaves two levels down)."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_layout_arithmetic():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "layout_check")
        subprocess.run([nvcc, "-std=c++17", "-O1", os.path.join(HERE, "layout_check.cu"), "-o", exe],
                       check=True, capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.stdout.strip() == "0" and r.returncode == 0, r.stdout + r.stderr
