"""Host-side check of the Zernike evaluation used by the kernels for bases
above N_p = 8 (paper_1608_04607_gb300/csrc/zernike_wide.h, the same function
the CUDA code runs): every basis index is produced once, and the values in
FP64 and FP32 match the oracle's factorial closed form (Sec. 3.1) up to
N_p = 20.  Compiles a small C++ program with the system compiler; no GPU
needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def zw_exe():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "zernike_wide_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1608_04607_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "zernike_wide_check.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("Np", [9, 14, 20])
def test_wide_zernike_matches_closed_form(oracle_mod, zw_exe, Np):
    rng = np.random.default_rng(Np)
    rho = np.sqrt(rng.uniform(0, 1, 300))
    phi = rng.uniform(0, 2 * np.pi, 300)
    pts = np.concatenate([np.stack([rho * np.cos(phi), rho * np.sin(phi)], 1),
                          [[0.0, 0.0], [1.0, 0.0], [0.0, -1.0], [0.6, 0.8]]])
    inp = f"{Np}\n" + "\n".join(f"{x:.17g} {y:.17g}" for x, y in pts) + "\n"
    out = subprocess.run([zw_exe], input=inp, capture_output=True, text=True, check=True)
    lines = out.stdout.strip().splitlines()
    assert len(lines) == 3 * len(pts)
    vals = np.array([[float(v) for v in s.split()] for s in lines]).reshape(len(pts), 3, -1)
    nb = (Np + 1) * (Np + 2) // 2
    assert vals.shape[2] == nb
    np.testing.assert_array_equal(vals[:, 2], 1.0)  # every index exactly once
    ref = oracle_mod.zernike(Np, pts[:, 0], pts[:, 1])
    # the closed form's alternating sums lose up to ~1e-10 at n = 20 near rho = 1
    np.testing.assert_allclose(vals[:, 0], ref, atol=1e-9, rtol=0)
    np.testing.assert_allclose(vals[:, 1], ref, atol=1e-5, rtol=0)
