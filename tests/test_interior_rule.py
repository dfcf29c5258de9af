"""Host-side check of the split polar rule for the interior-density face
integral (paper_1608_04607_gb300/csrc/interior_rule.cuh, the node generator
the CUDA kernel uses): its nodes, summed with the oracle's Zernike
polynomials, reproduce the oracle's adaptive cubature on the thin tets of the
768-tet cuboid and the solid angles of a thin tet.  Compiles a small C++
program with the system compiler; no GPU needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1608_04607_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rule_exe():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "interior_rule_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1608_04607_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "interior_rule_check.cpp"), "-o", exe], check=True)
    return exe


def _g_by_rule(exe, O, verts, tets, t, r, mu, Np, n):
    """g[4, nb] from the rule's nodes: sum w exp(-mu R) Z(dx, dy) / sqrt|F|."""
    e1, e2, nn = O.face_frames(verts, tets)
    area = O.face_areas(verts, tets)
    x, w = np.polynomial.legendre.leggauss(n)
    lines = [str(n), " ".join(f"{float(v):.17g}" for v in x), " ".join(f"{float(v):.17g}" for v in w)]
    for l in range(4):
        row = 4 * t + l
        P = verts[[tets[t, (l + 1 + k) % 4] for k in range(3)]]
        vals = list(P.reshape(-1)) + list(nn[row]) + list(e1[row]) + list(e2[row]) + list(r)
        lines.append(" ".join(f"{float(v):.17g}" for v in vals))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    nodes = np.array([[float(v) for v in s.split()] for s in out.stdout.strip().splitlines()])
    nodes = nodes.reshape(4, 6 * n * n, 4)
    g = np.zeros((4, (Np + 1) * (Np + 2) // 2))
    for l in range(4):
        wgt, R, dx, dy = nodes[l].T
        g[l] = (wgt * np.exp(-mu * R)) @ O.zernike(Np, dx, dy) / np.sqrt(area[4 * t + l])
    return g


def test_rule_nodes_match_the_adaptive_cubature(rule_exe, oracle_mod):
    m = inputs.kuhn_cuboid_mesh(4)
    mu = 0.4 * np.pi
    for t in (296, 343, 0):
        r = m.verts[m.tets[t]].mean(axis=0)
        g = _g_by_rule(rule_exe, oracle_mod, m.verts, m.tets, t, r, mu, 6, 24)
        ga, _ = oracle_mod.interior_g(m.verts, m.tets, t, r, mu, 6, nq=None)
        assert np.abs(g - ga).max() <= 1e-11 * np.abs(ga).max()
        gs = oracle_mod.interior_g_split(m.verts, m.tets, t, r, mu, 6, n=24)
        assert np.abs(g - gs).max() <= 1e-12 * np.abs(ga).max()  # same rule, written twice
    # centroid foot within 0.02 h of a face edge (jittered cube, log-normal damping)
    m = inputs.kuhn_cube_mesh(8, jitter=0.2, seed=0)
    mu_t = inputs.lognormal_mu(m)
    t = 1373
    r = m.verts[m.tets[t]].mean(axis=0)
    g = _g_by_rule(rule_exe, oracle_mod, m.verts, m.tets, t, r, float(mu_t[t]), 4, 24)
    ga, _ = oracle_mod.interior_g(m.verts, m.tets, t, r, float(mu_t[t]), 4, nq=None, rtol=1e-13)
    assert np.abs(g - ga).max() <= 1e-12 * np.abs(ga).max()


def test_rule_nodes_give_solid_angles(rule_exe, oracle_mod):
    verts = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.3, 0.3, 0.02]])
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    cen = verts.mean(axis=0)
    g = _g_by_rule(rule_exe, oracle_mod, verts, tets, 0, cen, 0.0, 2, 24)
    from test_oracle_source import _solid_angle

    for f in range(4):
        rho = oracle_mod.source_vector(verts, tets, [f], 2)
        p = verts[[tets[0, (f + 1 + k) % 4] for k in range(3)]]
        assert np.sum(g * rho) == pytest.approx(_solid_angle(cen, *p), rel=1e-9)
