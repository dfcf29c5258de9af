"""The seeded synthetic inputs: conforming positive-volume meshes, boundary
face counts, reproducible draws and the damping-field statistics."""
import numpy as np
import pytest

from paper_1608_04607_gb300 import inputs as I


@pytest.mark.parametrize("n", [1, 2, 5])
def test_kuhn_mesh_is_conforming(oracle_mod, n):
    m = I.kuhn_cube_mesh(n, jitter=0.2, seed=0)
    assert m.tets.shape == (6 * n ** 3, 4)
    a, b, c, d = (m.verts[m.tets[:, k]] for k in range(4))
    vol = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a) / 6
    assert vol.min() > 0
    assert vol.sum() == pytest.approx(1.0, rel=1e-12)  # tiles the unit cube
    topo = oracle_mod.topology(m.tets)
    assert topo.boundary.sum() == 12 * n * n
    bf = I.boundary_faces(m)
    np.testing.assert_array_equal(np.sort(bf[:, 0]), np.nonzero(topo.boundary)[0])


def test_sources_and_fields_are_reproducible():
    m = I.kuhn_cube_mesh(4)
    r1 = I.random_boundary_rows(m, 16, seed=2)
    r2 = I.random_boundary_rows(m, 16, seed=2)
    np.testing.assert_array_equal(r1, r2)
    mu = I.lognormal_mu(I.kuhn_cube_mesh(12), median=0.05, sigma=0.5, corr_cells=3)
    assert np.all(mu[0::6] == mu[5::6])  # six tets of a cell share the value
    z = np.log(mu[::6] / 0.05) / 0.5
    assert abs(np.mean(z)) < 0.5 and 0.3 < np.std(z) < 1.5
    s = I.source_row_minus_x(I.kuhn_cube_mesh(4), (0.5, 0.5))
    assert s in set(I.boundary_faces(I.kuhn_cube_mesh(4))[:, 0])


def test_kuhn_cuboid_mesh():
    from paper_1608_04607_gb300 import inputs as I

    m = I.kuhn_cuboid_mesh(3, length=2.0, jitter=0.2, seed=0)
    assert (m.nx, m.n, m.n_tets) == (6, 3, 6 * 6 * 9)
    v, t = m.verts, m.tets
    a, b, c, d = (v[t[:, k]] for k in range(4))
    vol = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a) / 6
    assert vol.min() > 0 and abs(vol.sum() - 2.0) < 1e-12
    assert np.allclose(v.min(0), [0, -0.5, -0.5]) and np.allclose(v.max(0), [2, 0.5, 0.5])
    rows = I.cuboid_rows_x0(m)
    assert rows.size == 2 * 3 * 3
    for r in rows:
        tt, f = divmod(int(r), 4)
        assert np.all(v[[t[tt, k] for k in range(4) if k != f], 0] == 0.0)
    assert np.array_equal(I.kuhn_cuboid_mesh(3).verts, m.verts)  # seeded
