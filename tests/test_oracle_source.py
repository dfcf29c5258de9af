"""Pins for the oracle's directed boundary sources (Sec. 4.1, Eq. RhoNeumann)
and per-tet interior densities (Eq. IntDens), and for the cuboid mesh.

The directed source is N_nm Z_n^m(p_d) sqrt|T|.  What fixes it independently
of the oracle's own code:
  - the normal-incidence projection the paper describes: only m = 0, even n
    survive, with Z_n^0(0) = (-1)^(n/2) and N_n0 = (n+1)/pi;
  - a face in the z = 0 plane whose frame is known by hand (e1 = x, e2 = y,
    n = z), where the coefficients follow from textbook low-order Zernike
    polynomials written out below;
  - rotation of d about the face normal by alpha multiplies a_(n,m) + i a_(n,-m)
    by exp(i m alpha) (a swapped e1/e2 or a sign error in m turns it the other way);
  - the mass of a combined source: the (0,0) coefficient of the unit-mass
    delta is sqrt|T|/pi on every face, whatever the direction (an isotropic
    unit density, of mass pi on the disc, has sqrt|T|).
The per-tet density is pinned on one tet with the source density itself
(no transport): for a unit isotropic density on a face and mu = 0, rho_T at a
point is the solid angle the face subtends there (Van Oosterom-Strackee).
"""
import numpy as np
import pytest

from paper_1608_04607_gb300 import inputs


def _area(verts, tets, r):
    t, f = divmod(int(r), 4)
    p = verts[[tets[t, (f + 1 + k) % 4] for k in range(3)]]
    return 0.5 * np.linalg.norm(np.cross(p[1] - p[0], p[2] - p[0]))


def test_normal_incidence_closed_form(oracle_mod):
    m = inputs.kuhn_cube_mesh(2, jitter=0.2, seed=0)
    rows = inputs.boundary_faces(m)[::7, 0]
    Np = 8
    x = oracle_mod.source_directed(m.verts, m.tets, rows, Np)
    for s, r in enumerate(rows):
        sa = np.sqrt(_area(m.verts, m.tets, r))
        for (n, mm) in oracle_mod.zernike_nm(Np):
            want = (n + 1) / np.pi * (-1) ** (n // 2) * sa if (mm == 0 and n % 2 == 0) else 0.0
            assert x[s, r, oracle_mod.zernike_index(n, mm)] == pytest.approx(want, abs=1e-13)
        others = np.delete(np.arange(m.n_rows), r)
        assert not np.any(x[s, others])


def test_textbook_low_orders_on_a_known_frame(oracle_mod):
    # face 3 of this tet is v0 v1 v2 in the z = 0 plane: e1 = x (first edge
    # v0 -> v1), n = +z (towards v3), e2 = n x e1 = y
    verts = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 1.5, 0.0], [0.3, 0.2, 1.0]])
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    th, ph = 0.6, 0.9
    d = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    x = oracle_mod.source_directed(verts, tets, [3], 4, dirs=[d])[0, 3]
    rho = np.sin(th)
    Z = {(0, 0): 1.0,
         (1, 1): rho * np.cos(ph), (1, -1): rho * np.sin(ph),
         (2, 0): 2 * rho ** 2 - 1, (2, 2): rho ** 2 * np.cos(2 * ph), (2, -2): rho ** 2 * np.sin(2 * ph),
         (3, 1): (3 * rho ** 3 - 2 * rho) * np.cos(ph), (3, -1): (3 * rho ** 3 - 2 * rho) * np.sin(ph),
         (3, 3): rho ** 3 * np.cos(3 * ph), (3, -3): rho ** 3 * np.sin(3 * ph),
         (4, 0): 6 * rho ** 4 - 6 * rho ** 2 + 1,
         (4, 2): (4 * rho ** 4 - 3 * rho ** 2) * np.cos(2 * ph), (4, -2): (4 * rho ** 4 - 3 * rho ** 2) * np.sin(2 * ph),
         (4, 4): rho ** 4 * np.cos(4 * ph), (4, -4): rho ** 4 * np.sin(4 * ph)}
    sa = np.sqrt(0.5 * 2.0 * 1.5)
    for (n, mm), z in Z.items():
        N = (2 * n + 2) / ((2.0 if mm == 0 else 1.0) * np.pi)
        assert x[oracle_mod.zernike_index(n, mm)] == pytest.approx(N * z * sa, abs=1e-13)


def test_rotation_about_the_normal(oracle_mod):
    m = inputs.kuhn_cube_mesh(2, jitter=0.2, seed=0)
    e1, e2, nn = oracle_mod.face_frames(m.verts, m.tets)
    Np, alpha = 6, 0.7
    rng = np.random.default_rng(4)
    for r in inputs.boundary_faces(m)[::11, 0]:
        n = nn[r]
        t = rng.normal(size=3)
        t -= (t @ n) * n
        d = 0.8 * n + 0.55 * t / np.linalg.norm(t)
        # Rodrigues rotation of d about n by alpha (right-handed)
        dr = d * np.cos(alpha) + np.cross(n, d) * np.sin(alpha) + n * (n @ d) * (1 - np.cos(alpha))
        a = oracle_mod.source_directed(m.verts, m.tets, [r], Np, dirs=[d])[0, r]
        b = oracle_mod.source_directed(m.verts, m.tets, [r], Np, dirs=[dr])[0, r]
        for nd in range(Np + 1):
            for mm in range(nd % 2, nd + 1, 2):
                if mm == 0:
                    assert b[oracle_mod.zernike_index(nd, 0)] == pytest.approx(a[oracle_mod.zernike_index(nd, 0)],
                                                                             abs=1e-12)
                    continue
                ca = a[oracle_mod.zernike_index(nd, mm)] + 1j * a[oracle_mod.zernike_index(nd, -mm)]
                cb = b[oracle_mod.zernike_index(nd, mm)] + 1j * b[oracle_mod.zernike_index(nd, -mm)]
                assert abs(cb - ca * np.exp(1j * mm * alpha)) < 1e-12


def test_combined_source_mass_and_rejection(oracle_mod):
    m = inputs.kuhn_cuboid_mesh(2, jitter=0.2, seed=0)
    rows = inputs.cuboid_rows_x0(m)
    x = oracle_mod.source_directed(m.verts, m.tets, rows, 4, combine=True)
    _, _, nn = oracle_mod.face_frames(m.verts, m.tets)
    assert x.shape == (m.n_rows, 15)
    for r in rows:
        assert x[r, 0] == pytest.approx(np.sqrt(_area(m.verts, m.tets, r)) / np.pi, abs=1e-14)
        assert nn[r] @ np.array([1.0, 0.0, 0.0]) == pytest.approx(1.0)  # x = 0 side: inward normal +x
    with pytest.raises(ValueError):
        oracle_mod.source_directed(m.verts, m.tets, rows[:1], 4, dirs=[-nn[rows[0]]])


def _solid_angle(r, a, b, c):
    """Van Oosterom-Strackee: solid angle of triangle abc seen from r."""
    A, B, C = a - r, b - r, c - r
    la, lb, lc = np.linalg.norm(A), np.linalg.norm(B), np.linalg.norm(C)
    num = abs(A @ np.cross(B, C))
    den = la * lb * lc + (A @ B) * lc + (A @ C) * lb + (B @ C) * la
    return 2.0 * np.arctan2(num, den)


def test_tet_density_of_an_isotropic_face_is_its_solid_angle(oracle_mod):
    m = inputs.kuhn_cube_mesh(1, jitter=0.0)
    Np = 3
    r = 4 * 2 + 1  # tet 2, face 1
    rho = oracle_mod.source_vector(m.verts, m.tets, [r], Np)  # unit isotropic density on the face
    dens = oracle_mod.tet_density(m.verts, m.tets, np.zeros(m.n_tets), Np, rho, nq=48)
    t, f = divmod(r, 4)
    cen = m.verts[m.tets[t]].mean(axis=0)
    p = m.verts[[m.tets[t, (f + 1 + k) % 4] for k in range(3)]]
    # rho_T(r) = Int cos / |r - s|^2 ds over the face = its solid angle from r;
    # the isotropic unit density has rho(s, p) = 1 for every direction
    assert dens[t] == pytest.approx(_solid_angle(cen, *p), rel=1e-9)
    assert np.count_nonzero(dens) == 1


def test_adaptive_interior_rule_on_a_thin_tet(oracle_mod):
    """A thin tet's centroid sits close to its base, where cos / R^2 peaks:
    the adaptive cubature still gives each face's solid angle (isotropic unit
    density, mu = 0), which a fixed 32-point rule misses by far more."""
    verts = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.3, 0.3, 0.02]])
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    cen = verts.mean(axis=0)
    for f in range(4):
        rho = oracle_mod.source_vector(verts, tets, [f], 2)
        p = verts[[tets[0, (f + 1 + k) % 4] for k in range(3)]]
        want = _solid_angle(cen, *p)
        got = oracle_mod.tet_density(verts, tets, np.zeros(1), 2, rho, nq=None)[0]
        assert got == pytest.approx(want, rel=1e-9)
        g, _ = oracle_mod.interior_g(verts, tets, 0, cen, 0.0, 2, nq=None)
        assert np.sum(g * rho) == pytest.approx(want, rel=1e-9)
    rho = oracle_mod.source_vector(verts, tets, [3], 2)
    fixed = oracle_mod.tet_density(verts, tets, np.zeros(1), 2, rho, nq=32)[0]
    assert abs(fixed - _solid_angle(cen, *verts[:3])) > 1e-6


def test_split_polar_interior_rule(oracle_mod):
    """The rule that splits each face at the foot of r and integrates in polar
    angles seen from r reproduces the adaptive cubature on the thin tets of the
    768-tet cuboid, where a 32 x 32 collapsed rule is off by percents, and the
    solid angles of the thin tet below."""
    m = inputs.kuhn_cuboid_mesh(4)
    mu = 0.4 * np.pi
    for t in (296, 343):
        r = m.verts[m.tets[t]].mean(axis=0)
        ga, _ = oracle_mod.interior_g(m.verts, m.tets, t, r, mu, 4, nq=None)
        gs = oracle_mod.interior_g_split(m.verts, m.tets, t, r, mu, 4, n=24)
        g32, _ = oracle_mod.interior_g(m.verts, m.tets, t, r, mu, 4, nq=32)
        s = np.abs(ga).max()
        assert np.abs(gs - ga).max() <= 1e-11 * s
        assert np.abs(g32 - ga).max() > 1e-3 * s
    # a jittered-cube tet whose centroid's foot lies within 0.02 h of a face
    # edge on two faces (an azimuth rule uniform in the angle is off by 4e-4
    # there with 24 points)
    m = inputs.kuhn_cube_mesh(8, jitter=0.2, seed=0)
    mu_t = inputs.lognormal_mu(m)
    t = 1373
    r = m.verts[m.tets[t]].mean(axis=0)
    ga, _ = oracle_mod.interior_g(m.verts, m.tets, t, r, float(mu_t[t]), 4, nq=None, rtol=1e-13)
    gs = oracle_mod.interior_g_split(m.verts, m.tets, t, r, float(mu_t[t]), 4, n=24)
    assert np.abs(gs - ga).max() <= 1e-12 * np.abs(ga).max()
    verts = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.3, 0.3, 0.02]])
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    cen = verts.mean(axis=0)
    g = oracle_mod.interior_g_split(verts, tets, 0, cen, 0.0, 2, n=24)
    for f in range(4):
        rho = oracle_mod.source_vector(verts, tets, [f], 2)
        p = verts[[tets[0, (f + 1 + k) % 4] for k in range(3)]]
        assert np.sum(g * rho) == pytest.approx(_solid_angle(cen, *p), rel=1e-9)
