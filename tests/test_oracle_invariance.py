"""Frame invariance of the observables (the face frame is a convention, Sec.
3.3 gives it only by example): reordering the vertices of every tet changes
every face's frame, its Zernike orientation, the linear spatial functions and
the numbering of rows, but not the physics, so the interior density at every
centroid (Eq. IntDens) of the solution for a physically fixed source must be
unchanged, for the piecewise-constant and the linear spatial basis and for an
isotropic and a normal-incidence source."""
import numpy as np
import pytest

from paper_1608_04607_gb300.inputs import kuhn_cube_mesh


def _row_of_face(tets, face_verts):
    """The row 4t + f whose face holds exactly the given three vertices."""
    key = set(int(v) for v in face_verts)
    for t in range(tets.shape[0]):
        for f in range(4):
            if set(int(tets[t, (f + 1 + k) % 4]) for k in range(3)) == key:
                return 4 * t + f
    raise AssertionError("face not found")


def _densities(oracle_mod, verts, tets, face, Np, spatial, mu, refl):
    """rho_T at every centroid for an isotropic and for a normal-incidence
    source on the given face, with fixed Gauss orders: order 32 per direction
    region (the regions are built from the tet's vertices by their roles, so
    both orderings meet the same nodes) and order 64 on each face for the
    density (the vertex order moves its nodes; order 32 leaves 2e-7 on the
    tets whose centroid is close to a face, order 64 1e-12)."""
    op = oracle_mod.assemble(verts, tets, np.full(tets.shape[0], mu), refl, Np, q=32, spatial=spatial)
    row = _row_of_face(tets, face)
    M = np.eye(op.nrows * op.nb) - oracle_mod.dense(op)
    out = []
    for rho0 in (oracle_mod.source_vector(verts, tets, [row], Np, spatial=spatial),
                 oracle_mod.source_directed(verts, tets, [row], Np, combine=True, spatial=spatial)):
        rho = np.linalg.solve(M, rho0.reshape(-1)).reshape(op.nrows, op.nb)
        out.append(oracle_mod.tet_density(verts, tets, np.full(tets.shape[0], mu), Np, rho, nq=64,
                                          spatial=spatial))
    return out


@pytest.mark.parametrize("spatial", [0, 1])
def test_interior_density_does_not_depend_on_vertex_order(oracle_mod, spatial):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=6)
    Np, mu, refl = 2, 0.6, 0.8
    # a boundary face on x = 0, named by its vertices
    topo = oracle_mod.topology(m.tets)
    cen = m.verts[m.tets].mean(axis=1)
    rows = [r for r in np.nonzero(topo.boundary)[0]
            if np.all(np.abs(m.verts[[m.tets[r // 4, (r % 4 + 1 + k) % 4] for k in range(3)], 0]) < 1e-12)]
    r0 = rows[0]
    face = [m.tets[r0 // 4, (r0 % 4 + 1 + k) % 4] for k in range(3)]
    ref = _densities(oracle_mod, m.verts, m.tets, face, Np, spatial, mu, refl)
    rng = np.random.default_rng(3)
    perm_tets = np.array([t[rng.permutation(4)] for t in m.tets], dtype=np.int32)
    assert np.allclose(cen, m.verts[perm_tets].mean(axis=1))
    got = _densities(oracle_mod, m.verts, perm_tets, face, Np, spatial, mu, refl)
    for g, r in zip(got, ref):
        assert np.abs(r).max() > 0
        np.testing.assert_allclose(g, r, rtol=0, atol=1e-10 * np.abs(r).max())
