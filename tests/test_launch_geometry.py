"""Host-side check of the pipelined applications' launch geometry
(paper_1608_04607_gb300/csrc/launch_geometry.h, shared with the CUDA code):
every bulk copy 16-byte aligned, shared memory within a block's limit, tile
rows and stages as the kernels require.  Compiles a small C++ program with
the system compiler; no GPU needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_launch_geometry_keeps_bulk_copies_aligned():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "geom_check")
    src = os.path.join(ROOT, "tests", "launch_geometry_check.cpp")
    inc = os.path.join(ROOT, "paper_1608_04607_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", inc, src, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok")
