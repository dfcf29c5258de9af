"""Pins for the oracle's linear spatial basis (the higher-order spatial
approximation the paper suggests in Sec. 3.1 and at the end of Sec. 4.1):
three orthonormal affine functions per face in place of the constant one.

- the basis is orthonormal on a triangle (numpy Gauss rule on the simplex);
- the blocks of the constant functions are the piecewise-constant operator;
- reciprocity between every test and trial function on one tet;
- conservation (Sec. 2): at mu = 0 with reflecting walls the mass row
  sum_I sqrt|T_I| B_(I,0,00),(J,s,nm) is sqrt|T_J| for (s, nm) = (0, 00) and 0
  for every other column, the linear functions carrying no mass;
- brute-force Monte Carlo ray tracing of whole blocks (5 sigma), the score
  weighted by the source function at the ray's start and the receiving
  function at its exit;
- the interior-density functional of the linear functions against a numpy
  collapsed Gauss rule of its definition (Eq. IntDens);
- sources of constant densities have no linear component (zero mean).
"""
import numpy as np
import pytest

from paper_1608_04607_gb300.inputs import kuhn_cube_mesh


def _jittered_tet():
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    return m.verts, m.tets[[9]].copy()


def _simplex_rule(n):
    x, w = np.polynomial.legendre.leggauss(n)
    u = 0.5 * (1 + x)
    U, Vv = np.meshgrid(u, u, indexing="ij")
    W = np.outer(w, w) * 0.25 * (1 - U)
    return U.ravel(), ((1 - U) * Vv).ravel(), W.ravel()  # l1, l2, weight (simplex area 1/2)


def test_linear_basis_is_orthonormal(oracle_mod):
    C = oracle_mod.p1_coeffs()
    l1, l2, w = _simplex_rule(8)
    L = np.stack([1 - l1 - l2, l1, l2])
    phi = C @ L  # sqrt|T| phi_a at the nodes
    G = (phi * w) @ phi.T * 2.0  # (1/|T|) Int phi_a phi_b
    np.testing.assert_allclose(G, np.eye(3), atol=1e-14)
    np.testing.assert_allclose(C[0], 1.0, atol=1e-15)  # the constant function comes first


def test_constant_functions_give_the_piecewise_constant_operator(oracle_mod):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    Np = 2
    topo = oracle_mod.topology(m.tets)
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    sel = np.isin(t, [0, 17, 40])
    mu = np.full(m.n_tets, 0.4)
    b1, d1, _, _ = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, mu, 0.8, Np, t[sel], f[sel], fp[sel], q=32,
                                               with_derivative=True, spatial=1)
    b0, d0, _, _ = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, mu, 0.8, Np, t[sel], f[sel], fp[sel], q=32,
                                               with_derivative=True)
    nz = oracle_mod.nbasis(Np)
    assert b1.shape[1:] == (3 * nz, 3 * nz)
    np.testing.assert_allclose(b1[:, :nz, :nz], b0, atol=1e-13)
    np.testing.assert_allclose(d1[:, :nz, :nz], d0, atol=1e-13)


@pytest.mark.parametrize("mu", [0.0, 0.8])
def test_reciprocity_linear_basis(oracle_mod, mu):
    V, T = _jittered_tet()
    Np = 3
    op = oracle_mod.assemble(V, T, np.array([mu]), 1.0, Np, q=32, spatial=1)
    N = np.tile(oracle_mod.zernike_invnorm(Np), 3)
    sign = np.tile(np.array([(-1) ** n for n, m in oracle_mod.zernike_nm(Np)]), 3)
    fps = {f: [k for k in range(4) if k != f] for f in range(4)}
    blk = lambda f, fp: op.blocks[f, fps[f].index(fp)]
    for f in range(4):
        for fp in range(4):
            if fp != f:
                lhs = blk(f, fp) / N[:, None]
                rhs = (blk(fp, f) / N[:, None]).T * np.outer(sign, sign)
                np.testing.assert_allclose(lhs, rhs, atol=1e-11)


def test_conservation_linear_basis(oracle_mod):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    Np = 2
    op = oracle_mod.assemble(m.verts, m.tets, np.zeros(m.n_tets), 1.0, Np, q=32, spatial=1)
    A = oracle_mod.face_areas(m.verts, m.tets)
    w = np.zeros((op.nrows, op.nb))
    w[:, 0] = np.sqrt(A)
    np.testing.assert_allclose(oracle_mod.apply(op, w, trans=True), w, atol=1e-11)


@pytest.mark.parametrize("pair", [(0, 1), (3, 2)])
def test_monte_carlo_linear_basis(oracle_mod, pair):
    V, T = _jittered_tet()
    f, fp = pair
    Np, mu, lam = 2, 0.7, 0.9
    topo = oracle_mod.topology(T)
    out, _, _, recv = oracle_mod.blocks_for_pairs(V, T, topo, np.array([mu]), lam, Np, np.array([0]),
                                                  np.array([f]), np.array([fp]), spatial=1)
    mean, se = oracle_mod.mc_block(V, T, 0, f, fp, int(recv[0]), mu, lam, Np, nsamp=4 * 10 ** 6, seed=3 + f,
                                   spatial=1)
    z = np.abs(out[0] - mean) / np.maximum(se, 1e-300)
    assert z.max() < 5.0, z.max()


def test_interior_density_linear_basis(oracle_mod):
    V, T = _jittered_tet()
    Np, mu = 3, 0.6
    r = V[T[0]].mean(axis=0)
    g, dg = oracle_mod.interior_g(V, T, 0, r, mu, Np, nq=None, spatial=1)
    nz = oracle_mod.nbasis(Np)
    g0, _ = oracle_mod.interior_g(V, T, 0, r, mu, Np, nq=None)
    np.testing.assert_allclose(g[:, :nz], g0, atol=1e-12 * np.abs(g0).max())
    # the definition on each face with a 64-point collapsed Gauss rule in numpy
    C = oracle_mod.p1_coeffs()
    l1, l2, w = _simplex_rule(64)
    e1, e2, nn = oracle_mod.face_frames(V, T)
    A = oracle_mod.face_areas(V, T)
    for l in range(4):
        P = V[[T[0, (l + 1 + k) % 4] for k in range(3)]]
        s = P[0] + np.outer(l1, P[1] - P[0]) + np.outer(l2, P[2] - P[0])
        rs = r - s
        R = np.linalg.norm(rs, axis=1)
        u = rs / R[:, None]
        ker = 2 * A[l] * w * (u @ nn[l]) * np.exp(-mu * R) / R ** 2
        Z = oracle_mod.zernike(Np, u @ e1[l], u @ e2[l])
        phi = C @ np.stack([1 - l1 - l2, l1, l2])
        ref = np.concatenate([(ker * phi[a]) @ Z for a in range(3)]) / np.sqrt(A[l])
        np.testing.assert_allclose(g[l], ref, atol=1e-10 * np.abs(ref).max())


def test_constant_densities_project_on_the_constant_function(oracle_mod):
    """A density constant over a face has no component along the linear
    functions (they have zero mean), so both sources of the linear basis are
    the constant basis' coefficients followed by zeros."""
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    topo = oracle_mod.topology(m.tets)
    rows = np.nonzero(topo.boundary)[0][:5]
    Np = 3
    nz = oracle_mod.nbasis(Np)
    e1, e2, nn = oracle_mod.face_frames(m.verts, m.tets)
    dirs = nn[rows] + 0.3 * e1[rows] - 0.2 * e2[rows]
    for p0, p1 in ((oracle_mod.source_vector(m.verts, m.tets, rows, Np),
                    oracle_mod.source_vector(m.verts, m.tets, rows, Np, spatial=1)),
                   (oracle_mod.source_directed(m.verts, m.tets, rows, Np, dirs=dirs),
                    oracle_mod.source_directed(m.verts, m.tets, rows, Np, dirs=dirs, spatial=1))):
        assert p1.shape[-1] == 3 * nz
        np.testing.assert_array_equal(p1[..., :nz], p0)
        assert not np.any(p1[..., nz:])
