"""Pins for the oracle's direction regions and spatial integral (Sec. 3.3-3.4).

- the seven direction regions tile the hemisphere: their projected solid
  angles sum to pi, and each equals Lambert's closed form for a spherical
  polygon, 1/2 sum_k gamma_k (nu_k . n);
- the three regions where P falls beyond the shared edge BC or at B, C give an
  empty integration triangle (Sec. 3.3);
- for every direction the clipped areas over the three destination faces
  partition the source face, and each damped area equals the paper's closed
  form h|BC|/(mu L)^2 (mu L - 1 + exp(-mu L)) with O found by the paper's
  seven-region construction (Sec. 3.3);
- brute-force ray tracing of a dense point grid agrees with the clipping.
"""
import numpy as np
import pytest

from paper_1608_04607_gb300.inputs import kuhn_cube_mesh

REGION_GENS = {
    0: lambda A, B, C, D: [D - A, D - B, D - C],
    1: lambda A, B, C, D: [D - A, B - A, C - A],
    2: lambda A, B, C, D: [D - A, D - B, C - B, C - A],
    3: lambda A, B, C, D: [D - A, D - C, B - C, B - A],
    4: lambda A, B, C, D: [D - B, C - B, A - B],
    5: lambda A, B, C, D: [D - C, A - C, B - C],
    6: lambda A, B, C, D: [D - B, D - C, A - C, A - B],
}


def _face(V, tv, f):
    p = [V[tv[(f + 1 + k) % 4]] for k in range(3)]
    apex = V[tv[f]]
    c = np.cross(p[1] - p[0], p[2] - p[0])
    if np.dot(c, apex - p[0]) < 0:
        c = -c
    return p, apex, c / np.linalg.norm(c)


def _lambert(gens, n):
    u = [g / np.linalg.norm(g) for g in gens]
    phi = np.zeros(3)
    for k in range(len(u)):
        a, b = u[k], u[(k + 1) % len(u)]
        cr = np.cross(a, b)
        gamma = np.arctan2(np.linalg.norm(cr), np.dot(a, b))
        phi += 0.5 * gamma * cr / np.linalg.norm(cr)
    return abs(np.dot(phi, n))


@pytest.fixture(scope="module")
def mesh():
    return kuhn_cube_mesh(3, jitter=0.2, seed=5)


def test_regions_tile_hemisphere_and_match_lambert(oracle_mod, mesh):
    V, T = mesh.verts, mesh.tets
    for t in (0, 17, 58, 101):
        tv = T[t]
        for f in range(4):
            p, D, n = _face(V, tv, f)
            for fp in range(4):
                if fp == f:
                    continue
                A = V[tv[fp]]
                B, C = [V[tv[k]] for k in range(4) if k not in (f, fp)]
                tot = 0.0
                for r in range(7):
                    s = oracle_mod.region_cos_measure(V, T, t, f, fp, r, q=64)
                    assert s == pytest.approx(_lambert(REGION_GENS[r](A, B, C, D), n), rel=1e-9, abs=1e-12)
                    tot += s
                assert tot == pytest.approx(np.pi, abs=1e-10)


def test_empty_regions_give_zero(oracle_mod, mesh):
    V, T = mesh.verts, mesh.tets
    topo = oracle_mod.topology(T)
    t, f, fp = oracle_mod.pair_list(T.shape[0])
    sel = np.arange(24, 48)
    out, _, _, _ = oracle_mod.blocks_for_pairs(V, T, topo, np.full(T.shape[0], 0.3), 1.0, 3, t[sel], f[sel], fp[sel],
                                               q=16, regions_mask=0x70)
    assert np.abs(out).max() < 1e-12
    full, _, _, _ = oracle_mod.blocks_for_pairs(V, T, topo, np.full(T.shape[0], 0.3), 1.0, 3, t[sel], f[sel],
                                                fp[sel], q=16, regions_mask=0x7F)
    part, _, _, _ = oracle_mod.blocks_for_pairs(V, T, topo, np.full(T.shape[0], 0.3), 1.0, 3, t[sel], f[sel],
                                                fp[sel], q=16, regions_mask=0x0F)
    np.testing.assert_allclose(full, part, atol=1e-13)


def _paper_O_construction(A, B, C, D, n, d):
    """Sec. 3.3: P is where the line through D along d meets the source plane;
    its region among the seven cut out by lines AB, BC, CA gives O, and the
    integration triangle is OBC.  Returns (area(OBC), L_max) or (0, 0)."""
    e1 = (B - A) / np.linalg.norm(B - A)
    e2 = np.cross(n, e1)
    to2 = lambda X: np.array([np.dot(X - A, e1), np.dot(X - A, e2)])
    a, b, c = to2(A), to2(B), to2(C)
    D3 = np.dot(D - A, n)
    t = D3 / np.dot(d, n)
    P3 = D - t * d
    P = to2(P3)

    def side(X, Y, Z, Q):  # >= 0 when Q is on Z's side of line XY
        cr = lambda u, v: u[0] * v[1] - u[1] * v[0]
        return cr(Y - X, Q - X) * np.sign(cr(Y - X, Z - X))

    sBC, sCA, sAB = side(b, c, a, P), side(c, a, b, P), side(a, b, c, P)
    if sBC <= 0:
        return 0.0, 0.0  # P beyond BC or in the wedges at B, C: empty
    if sCA >= 0 and sAB >= 0:
        O = P
    elif sCA < 0 and sAB < 0:
        O = a
    elif sAB < 0:  # strip on AB: O = AB intersect PC
        M = np.column_stack([b - a, c - P])
        s, _ = np.linalg.solve(M, c - a)
        O = a + s * (b - a)
    else:  # strip on CA: O = CA intersect PB
        M = np.column_stack([c - a, b - P])
        s, _ = np.linalg.solve(M, b - a)
        O = a + s * (c - a)
    cr = lambda u, v: u[0] * v[1] - u[1] * v[0]
    area = 0.5 * abs(cr(b - O, c - O))
    # L is affine on the plane, zero on BC, |PD| at P; the longest ray leaves from O
    dist_bc = lambda Q: abs(cr(c - b, Q - b)) / np.linalg.norm(c - b)
    Lmax = t * dist_bc(O) / dist_bc(P)
    return area, Lmax


def test_spatial_matches_paper_closed_form(oracle_mod, mesh):
    V, T = mesh.verts, mesh.tets
    rng = np.random.default_rng(4)
    for t in (3, 44, 90):
        tv = T[t]
        for f in range(4):
            p, D, n = _face(V, tv, f)
            area_f = 0.5 * np.linalg.norm(np.cross(p[1] - p[0], p[2] - p[0]))
            for _ in range(40):
                # random inward direction (includes near-grazing ones)
                v = rng.normal(size=3)
                v -= np.dot(v, n) * n
                v /= np.linalg.norm(v)
                ct = rng.uniform(0.02, 1.0)
                d = ct * n + np.sqrt(1 - ct * ct) * v
                for mu in (0.0, 2.5):
                    S, dS, Aclip = oracle_mod.spatial(V, T, t, f, d, mu)
                    assert Aclip.sum() == pytest.approx(area_f, rel=1e-12)
                    fps = [k for k in range(4) if k != f]
                    for k, fp in enumerate(fps):
                        A = V[tv[fp]]
                        B, C = [V[tv[j]] for j in range(4) if j not in (f, fp)]
                        a_nab, Lm = _paper_O_construction(A, B, C, D, n, d)
                        assert Aclip[k] == pytest.approx(a_nab, rel=1e-9, abs=1e-13)
                        x = mu * Lm
                        closed = a_nab if x == 0 else 2 * a_nab * (x - 1 + np.exp(-x)) / x ** 2
                        assert S[k] == pytest.approx(closed, rel=1e-9, abs=1e-13)


def test_spatial_vs_raytrace(oracle_mod, mesh):
    V, T = mesh.verts, mesh.tets
    t, f = 7, 2
    tv = T[t]
    p, D, n = _face(V, tv, f)
    faces = {k: _face(V, tv, k) for k in range(4)}
    N = 300
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    keep = i + j < N
    u = (i[keep] + 1 / 3) / N
    w = (j[keep] + 1 / 3) / N
    pts = p[0] + np.outer(u, p[1] - p[0]) + np.outer(w, p[2] - p[0])
    # the upside-down sub-triangles
    keep2 = i + j < N - 1
    u2 = (i[keep2] + 2 / 3) / N
    w2 = (j[keep2] + 2 / 3) / N
    pts = np.vstack([pts, p[0] + np.outer(u2, p[1] - p[0]) + np.outer(w2, p[2] - p[0])])
    area_f = 0.5 * np.linalg.norm(np.cross(p[1] - p[0], p[2] - p[0]))
    wt = area_f / (N * N)
    d = np.array([0.3, -0.2, 0.0]) + n
    d /= np.linalg.norm(d)
    mu = 1.5
    best = np.full(len(pts), np.inf)
    ex = np.full(len(pts), -1)
    for k in range(4):
        if k == f:
            continue
        pk, _, nk = faces[k]
        dn = -np.dot(d, nk)
        if dn <= 0:
            continue
        tk = ((pts - pk[0]) @ nk) / dn
        better = tk < best
        best[better] = tk[better]
        ex[better] = k
    S, _, Aclip = oracle_mod.spatial(V, T, t, f, d, mu)
    for idx, k in enumerate([k for k in range(4) if k != f]):
        sel = ex == k
        assert wt * sel.sum() == pytest.approx(Aclip[idx], rel=2e-2, abs=2e-3 * area_f)
        assert wt * np.exp(-mu * best[sel]).sum() == pytest.approx(S[idx], rel=2e-2, abs=2e-3 * area_f)
