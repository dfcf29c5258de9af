"""Pins for the oracle's point source (Sec. 4.2, Eq. SourceRho):

- all power leaves the source: with mu = 0 the flux-weighted (0,0)
  coefficients sum to 4 strength (the full sphere, 4 pi, over the pi of the
  (0,0) normalisation), for a source inside a tet, on an interior face, on an
  interior edge and at an interior vertex (where 24 Kuhn tets share it); on
  the cube's surface half the sphere points out of the mesh;
- each face's (0,0) coefficient is strength * solid angle / (pi sqrt|F|), the
  solid angle by Van Oosterom-Strackee;
- with damping, the total equals 4 strength E[exp(-mu R(u))] over uniform
  directions u, R(u) the distance to the tet's boundary along u, estimated by
  sampling directions and intersecting face planes (a separate method);
- at the centroid of a regular tetrahedron every face sees the same (0,0)
  value, and the 3-fold symmetry of each face about the source's foot point
  makes the (1,+-1) and (2,+-2) moments vanish while (3,+-3) does not.
"""
import numpy as np
import pytest

from paper_1608_04607_gb300.inputs import kuhn_cube_mesh

REG_V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
ONE_TET = np.array([[0, 1, 2, 3]], dtype=np.int32)


def _solid_angle(r, a, b, c):
    A, B, C = a - r, b - r, c - r
    la, lb, lc = np.linalg.norm(A), np.linalg.norm(B), np.linalg.norm(C)
    num = abs(A @ np.cross(B, C))
    den = la * lb * lc + (A @ B) * lc + (A @ C) * lb + (B @ C) * la
    return 2.0 * np.arctan2(num, den)


@pytest.fixture(scope="module")
def mesh():
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    return m.verts, m.tets


def _points(V, T):
    """A point inside tet 20, on an interior face of it, on an edge of it that
    is not on the cube's surface, and the interior grid vertex (1, 1, 1)."""
    tv = V[T[20]]
    inner = lambda x: np.all((x > 1e-9) & (x < 1 - 1e-9))  # noqa: E731
    face = next(tv[[k for k in range(4) if k != l]].mean(axis=0) for l in range(4)
                if inner(tv[[k for k in range(4) if k != l]].mean(axis=0)))
    edge = next((tv[i] + tv[j]) / 2 for i in range(4) for j in range(i + 1, 4) if inner((tv[i] + tv[j]) / 2))
    vid = 1 + 3 * (1 + 3 * 1)
    return {"inside": tv.mean(axis=0), "face": face, "edge": edge, "vertex": V[vid]}


@pytest.mark.parametrize("where", ["inside", "face", "edge", "vertex"])
def test_all_power_leaves_the_source(oracle_mod, mesh, where):
    V, T = mesh
    r0 = _points(V, T)[where]
    a = oracle_mod.point_source(V, T, r0, 3, np.zeros(T.shape[0]), 1.0, strength=2.5)
    A = oracle_mod.face_areas(V, T)
    assert np.sum(np.sqrt(A) * a[:, 0]) == pytest.approx(4 * 2.5, rel=1e-10)


def test_a_source_on_the_surface_sends_half(oracle_mod, mesh):
    V, T = mesh
    topo = oracle_mod.topology(T)
    row = int(np.nonzero(topo.boundary)[0][3])
    t, l = divmod(row, 4)
    r0 = V[[T[t, (l + 1 + k) % 4] for k in range(3)]].mean(axis=0)
    a = oracle_mod.point_source(V, T, r0, 2, np.zeros(T.shape[0]), 1.0)
    A = oracle_mod.face_areas(V, T)
    assert np.sum(np.sqrt(A) * a[:, 0]) == pytest.approx(2.0, rel=1e-10)


def test_face_values_are_solid_angles(oracle_mod, mesh):
    V, T = mesh
    r0 = _points(V, T)["inside"]
    a = oracle_mod.point_source(V, T, r0, 2, np.zeros(T.shape[0]), 1.0)
    topo = oracle_mod.topology(T)
    A = oracle_mod.face_areas(V, T)
    for l in range(4):
        row = 4 * 20 + l
        p = V[[T[20, (l + 1 + k) % 4] for k in range(3)]]
        rec = int(topo.recv[row])
        assert a[rec, 0] == pytest.approx(_solid_angle(r0, *p) / (np.pi * np.sqrt(A[row])), rel=1e-10)


def test_damped_total_by_sampled_directions(oracle_mod, mesh):
    V, T = mesh
    r0 = _points(V, T)["inside"]
    mu = 1.7
    a = oracle_mod.point_source(V, T, r0, 1, np.full(T.shape[0], mu), 1.0)
    A = oracle_mod.face_areas(V, T)
    total = np.sum(np.sqrt(A) * a[:, 0])
    # exit distance of uniform directions from r0 through tet 20's face planes
    rng = np.random.default_rng(1)
    u = rng.standard_normal((400000, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    P = V[T[20]]
    dist = np.full(u.shape[0], np.inf)
    for l in range(4):
        q = P[[(l + 1 + k) % 4 for k in range(3)]]
        n = np.cross(q[1] - q[0], q[2] - q[0])
        n /= np.linalg.norm(n)
        if (P[l] - q[0]) @ n > 0:
            n = -n  # outward
        un = u @ n
        t = np.where(un > 0, ((q[0] - r0) @ n) / np.where(un > 0, un, 1.0), np.inf)
        dist = np.minimum(dist, t)
    e = np.exp(-mu * dist)
    est, se = 4 * e.mean(), 4 * e.std() / np.sqrt(e.size)
    assert abs(total - est) < 5 * se, (total, est, se)
    assert total < 4.0


def test_regular_tet_centroid_symmetry(oracle_mod):
    a = oracle_mod.point_source(REG_V, ONE_TET, REG_V.mean(axis=0), 3, np.zeros(1), 1.0)
    A = oracle_mod.face_areas(REG_V, ONE_TET)
    idx = oracle_mod.zernike_index
    np.testing.assert_allclose(a[:, 0], 1.0 / np.sqrt(A), rtol=1e-12)  # a quarter of the sphere each
    for m in (1, -1):
        np.testing.assert_allclose(a[:, idx(1, m)], 0.0, atol=1e-13)
        np.testing.assert_allclose(a[:, idx(3, m)], 0.0, atol=1e-13)
    for m in (2, -2):
        np.testing.assert_allclose(a[:, idx(2, m)], 0.0, atol=1e-13)
    assert np.all(np.hypot(a[:, idx(3, 3)], a[:, idx(3, -3)]) > 1e-3)


def test_rays_arrive_pointing_away_from_the_source(oracle_mod):
    """Off-centre source: on a face, the mean tangential direction of the arriving
    rays (the (1,+-1) moments) points from the source's foot on the face plane
    towards the face, i.e. along the weighted mean of s - foot (a reversed ray
    direction would point the other way)."""
    r0 = REG_V.mean(axis=0) + 0.45 * (REG_V[0] - REG_V.mean(axis=0))  # towards vertex 0
    a = oracle_mod.point_source(REG_V, ONE_TET, r0, 1, np.zeros(1), 1.0)
    e1, e2, nn = oracle_mod.face_frames(REG_V, ONE_TET)
    idx = oracle_mod.zernike_index
    for l in (1, 2, 3):  # faces that hold vertex 0
        p = REG_V[[ONE_TET[0, (l + 1 + k) % 4] for k in range(3)]]
        foot = r0 - ((r0 - p[0]) @ nn[l]) * nn[l]
        away = p.mean(axis=0) - foot  # the face lies mostly on this side of the foot
        got = np.array([a[l, idx(1, 1)], a[l, idx(1, -1)]])
        want = np.array([away @ e1[l], away @ e2[l]])
        cos = got @ want / (np.linalg.norm(got) * np.linalg.norm(want))
        assert cos > 0.9, (l, cos)
