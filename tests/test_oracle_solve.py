"""Pins for the oracle's stationary solve (Sec. 2, Eqs. NSum and GovIE) and the
adjoint gradient of the interior-density functional (Sec. 4.1, Eq. IntDens).

- the Neumann series, dense LU and GMRES give the same rho;
- the discrete balance identity w^T (I - B) rho = w^T rho0 (w the mass weights);
- the interior density kernel integrates to solid angles: at mu = 0,
  sqrt|T_l| g_(l,00)(r) is the solid angle of face l seen from r (Van
  Oosterom-Strackee closed form) and the four faces sum to 4 pi;
- the adjoint identity lam^T rho0 = g^T rho with (I - B)^T lam = g;
- dJ/dmu by the adjoint equals central finite differences of J.
"""
import numpy as np
import pytest

from paper_1608_04607_gb300.inputs import kuhn_cube_mesh, workload, uniform_mu


def test_config_small_neumann_lu_gmres(oracle_mod):
    w = workload("kuhn1_np2")
    m = w["mesh"]
    op = oracle_mod.assemble(m.verts, m.tets, w["mu"], w["refl"], w["Np"])
    assert np.all(op.q_used > 0)
    rho0 = oracle_mod.source_vector(m.verts, m.tets, w["sources"], w["Np"])
    x_lu = oracle_mod.solve_dense(op, rho0)
    x_ne, it = oracle_mod.neumann(op, rho0, tol=1e-13)
    assert it > 0
    x_gm, itg = oracle_mod.solve_gmres(op, rho0, tol=1e-13)
    assert itg > 0
    np.testing.assert_allclose(x_ne, x_lu, rtol=0, atol=1e-11 * np.abs(x_lu).max())
    np.testing.assert_allclose(x_gm, x_lu, rtol=0, atol=1e-11 * np.abs(x_lu).max())
    # mass balance: w^T (I - B) x = w^T rho0
    A = oracle_mod.face_areas(m.verts, m.tets)
    wv = np.zeros_like(rho0)
    wv[:, 0] = np.sqrt(A)
    lhs = np.sum(wv * (x_lu - oracle_mod.apply(op, x_lu)))
    assert lhs == pytest.approx(np.sum(wv * rho0), rel=1e-12)
    # damping and partial reflection: the spectral radius is below one
    M = oracle_mod.dense(op)
    assert np.max(np.abs(np.linalg.eigvals(M))) < 1.0


def _solid_angle(r, a, b, c):
    a, b, c = a - r, b - r, c - r
    la, lb, lc = np.linalg.norm(a), np.linalg.norm(b), np.linalg.norm(c)
    num = abs(np.dot(a, np.cross(b, c)))
    den = la * lb * lc + np.dot(a, b) * lc + np.dot(a, c) * lb + np.dot(b, c) * la
    return 2 * np.arctan2(num, den)


def test_interior_kernel_solid_angles(oracle_mod):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    A = oracle_mod.face_areas(m.verts, m.tets)
    for t in (0, 13, 40):
        tv = m.tets[t]
        cen = m.verts[tv].mean(axis=0)
        # the kernel 1/|r - s|^2 is smooth on every face for interior r; the
        # collapsed Gauss rule converges fast at the centroid, slower near a face
        for r, rel in ((cen, 1e-10), (0.8 * cen + 0.2 * m.verts[tv[2]], 1e-7)):
            g, _ = oracle_mod.interior_g(m.verts, m.tets, t, r, 0.0, 2, nq=40)
            total = 0.0
            for l in range(4):
                tri = [m.verts[tv[(l + 1 + k) % 4]] for k in range(3)]
                om = _solid_angle(r, *tri)
                assert np.sqrt(A[4 * t + l]) * g[l, 0] == pytest.approx(om, rel=rel)
                total += om
            assert total == pytest.approx(4 * np.pi, rel=1e-12)  # closed form


def _small_problem(oracle_mod, mu):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    Np = 2
    op = oracle_mod.assemble(m.verts, m.tets, mu, 0.8, Np, q=16, with_derivative=True)
    rows = np.array([1, 9])  # any rows work for the identities; use boundary ones
    topo = oracle_mod.topology(m.tets)
    rows = np.nonzero(topo.boundary)[0][[0, 7]]
    rho0 = oracle_mod.source_vector(m.verts, m.tets, rows, Np)
    receiver = np.array([20, 21, 30])
    return m, Np, op, rho0, receiver


def test_adjoint_identity_and_fd(oracle_mod):
    rng = np.random.default_rng(5)
    m0 = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    mu = rng.uniform(0.2, 0.6, m0.n_tets)
    m, Np, op, rho0, receiver = _small_problem(oracle_mod, mu)
    rho = oracle_mod.solve_dense(op, rho0)
    gvec, dg = oracle_mod.receiver_functional(m.verts, m.tets, mu, Np, receiver)
    lam, _ = oracle_mod.solve_gmres(op, gvec, tol=1e-14, trans=True)
    assert np.sum(lam * rho0) == pytest.approx(np.sum(gvec * rho), rel=1e-11)
    grad = oracle_mod.gradient(op, rho, lam, dg, m.n_tets)

    def J(mu_vec):
        o = oracle_mod.assemble(m.verts, m.tets, mu_vec, 0.8, Np, q=16)
        r = oracle_mod.solve_dense(o, rho0)
        gv, _ = oracle_mod.receiver_functional(m.verts, m.tets, mu_vec, Np, receiver)
        return float(np.sum(gv * r))

    h = 1e-4
    for e in (0, 20, 31, 47):
        mp, mm = mu.copy(), mu.copy()
        mp[e] += h
        mm[e] -= h
        fd = (J(mp) - J(mm)) / (2 * h)
        assert grad[e] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(grad).max())


def test_dblocks_match_fd(oracle_mod):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    topo = oracle_mod.topology(m.tets)
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    sel = np.arange(0, 60, 7)
    mu = np.full(m.n_tets, 0.4)
    _, db, _, _ = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, mu, 0.9, 3, t[sel], f[sel], fp[sel], q=16,
                                              with_derivative=True)
    h = 1e-5
    bp, _, _, _ = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, mu + h, 0.9, 3, t[sel], f[sel], fp[sel], q=16)
    bm, _, _, _ = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, mu - h, 0.9, 3, t[sel], f[sel], fp[sel], q=16)
    np.testing.assert_allclose(db, (bp - bm) / (2 * h), atol=1e-9)
