"""Host-side check of the closed-form spatial matrix of the linear spatial
basis (paper_1608_04607_gb300/csrc/p1_basis.h, the function the CUDA
assembly runs): for directions in every non-empty region of Sec. 3.3, on
boundary and interior face pairs, the GPU's matrix M[b][a] (moments of the
damping over the visible triangle OBC against the barycentric products of the
two faces' functions) matches the oracle's clipping and Gauss integration of
the same integral.  The inputs s_X = d_z beta_X(P), |OBC| and L_O are formed
here from the geometry as the assembly forms them.  Compiles a small C++
program with the system compiler; no GPU needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1608_04607_gb300.inputs import kuhn_cube_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def p1_exe():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "p1_spatial_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1608_04607_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "p1_spatial_check.cpp"), "-o", exe], check=True)
    return exe


def _inputs(oracle_mod, m, topo, t, f, fp, d, mu):
    """(sA, sB, sC, d_z, |OBC|, mu L_O, positions) of direction d, or None when
    no source point sees face fp (s_A <= 0)."""
    e1, e2, nn = oracle_mod.face_frames(m.verts, m.tets)
    row = 4 * t + f
    tv = m.tets[t]
    order = [(f + 1 + k) % 4 for k in range(3)]  # the source face's frame order
    p0 = m.verts[tv[order[0]]]
    loc = lambda v: np.array([(v - p0) @ e1[row], (v - p0) @ e2[row], (v - p0) @ nn[row]])
    bc = [v for v in order if v != fp]
    A, B, C, Dv = (loc(m.verts[tv[v]]) for v in (fp, bc[0], bc[1], f))
    dl = np.array([d @ e1[row], d @ e2[row], d @ nn[row]])
    P = Dv - Dv[2] / dl[2] * dl  # the apex projected along -d onto the source plane
    T2 = np.array([[A[0], B[0], C[0]], [A[1], B[1], C[1]], [1.0, 1.0, 1.0]])
    beta = np.linalg.solve(T2, np.array([P[0], P[1], 1.0]))
    sA, sB, sC = dl[2] * beta
    if sA <= 0:
        return None
    den = sA + max(sB, 0.0) + max(sC, 0.0)
    u, v = B[:2] - A[:2], C[:2] - A[:2]
    area = 0.5 * abs(u[0] * v[1] - u[1] * v[0])
    R = int(topo.recv[4 * t + fp])
    rt, rf = R // 4, R % 4
    rorder = [m.tets[rt, (rf + 1 + k) % 4] for k in range(3)]
    pos = [order.index(fp), order.index(bc[0]), order.index(bc[1]),
           rorder.index(tv[bc[0]]), rorder.index(tv[bc[1]]), rorder.index(tv[f])]
    return (sA, sB, sC, dl[2], area * sA / den, mu * Dv[2] / den, pos, R)


@pytest.mark.parametrize("mu", [0.0, 0.7, 9.0, 40.0])
def test_closed_form_matches_clipping(oracle_mod, p1_exe, mu):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    topo = oracle_mod.topology(m.tets)
    e1, e2, nn = oracle_mod.face_frames(m.verts, m.tets)
    rng = np.random.default_rng(int(mu * 10) + 1)
    cen = m.verts[m.tets].mean(axis=1)
    inner = int(np.argmin(np.abs(cen - 0.5).max(axis=1)))
    cases = []
    for t in (9, inner):
        for f in range(4):
            row = 4 * t + f
            for fp in [k for k in range(4) if k != f]:
                for _ in range(12):
                    # cosine-weighted inward direction
                    px, py = rng.uniform(-1, 1, 2)
                    if px * px + py * py >= 1:
                        continue
                    d = px * e1[row] + py * e2[row] + np.sqrt(1 - px * px - py * py) * nn[row]
                    inp = _inputs(oracle_mod, m, topo, t, f, fp, d, mu)
                    if inp is not None:
                        cases.append((t, f, fp, d, inp))
    assert len(cases) > 60
    lines = [" ".join(f"{float(v):.9g}" for v in c[4][:6]) + " " + " ".join(str(k) for k in c[4][6]) for c in cases]
    out = subprocess.run([p1_exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    got = np.array([[float(v) for v in s.split()] for s in out.stdout.strip().splitlines()]).reshape(-1, 3, 3)
    for (t, f, fp, d, inp), M in zip(cases, got):
        S, _ = oracle_mod.spatial_p1(m.verts, m.tets, t, f, fp, inp[7], d, mu, nq=16)
        scale = max(abs(S[0, 0]), 1e-300)  # the damped visible area
        assert np.abs(M - S).max() <= 2e-5 * scale, (t, f, fp, M, S)
