"""Pins for whole operator blocks of the oracle (Sec. 3.2, Eqs. Bapprox/B4DInt).

- regular tetrahedron at mu = 0: every face sees each other face with view
  factor 1/3 (symmetry plus closure), so B_(00),(00) = 1/3 for all 12 pairs;
- reciprocity: reversing a ray swaps source and receiving face and negates
  both tangential momenta, so on one tet with lambda = 1,
  B_{(l',n'm'),(l,nm)} / N_{n'm'} = (-1)^(n+n') B_{(l,nm),(l',n'm')} / N_{nm};
- brute-force Monte Carlo ray tracing of individual blocks (5 sigma);
- view factors (the (0,0) entries at mu = 0) against the contour-integral
  (Stokes) form on a jittered tet;
- conservation (Sec. 2): with mu = 0 and fully reflecting walls the phase-space
  mass pi sum_J sqrt|T_J| rho_(J,00) is preserved, i.e. w^T B = w^T with
  w_I = sqrt|T_I| on the (0,0) slots and 0 elsewhere;
- the adaptive order doubling reaches its tolerance.
"""
import numpy as np
import pytest

from paper_1608_04607_gb300.inputs import kuhn_cube_mesh

REG_V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
ONE_TET = np.array([[0, 1, 2, 3]], dtype=np.int32)


def test_regular_tet_view_factor(oracle_mod):
    op = oracle_mod.assemble(REG_V, ONE_TET, np.array([0.0]), 1.0, 2, q=32)
    np.testing.assert_allclose(op.blocks[:, :, 0, 0], 1.0 / 3.0, atol=1e-12)


def _jittered_tet():
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    return m.verts, m.tets[[9]].copy()


@pytest.mark.parametrize("mu", [0.0, 0.8])
def test_reciprocity_single_tet(oracle_mod, mu):
    V, T = _jittered_tet()
    Np = 3
    op = oracle_mod.assemble(V, T, np.array([mu]), 1.0, Np, q=32)
    N = oracle_mod.zernike_invnorm(Np)
    sign = np.array([(-1) ** n for n, m in oracle_mod.zernike_nm(Np)])
    fps = {f: [k for k in range(4) if k != f] for f in range(4)}
    blk = lambda f, fp: op.blocks[f, fps[f].index(fp)]
    for f in range(4):
        for fp in range(4):
            if fp == f:
                continue
            lhs = blk(f, fp) / N[:, None]
            rhs = (blk(fp, f) / N[:, None]).T * np.outer(sign, sign)
            np.testing.assert_allclose(lhs, rhs, atol=1e-11)
    # view factor closure at mu = 0: sum_l' sqrt(A_l'/A_l) B_00,00 = 1
    if mu == 0.0:
        A = oracle_mod.face_areas(V, T)
        for f in range(4):
            s = sum(np.sqrt(A[fp] / A[f]) * blk(f, fp)[0, 0] for fp in fps[f])
            assert s == pytest.approx(1.0, abs=1e-11)


@pytest.mark.parametrize("pair", [(0, 1), (2, 3), (3, 0)])
def test_monte_carlo_ray_tracing(oracle_mod, pair):
    V, T = _jittered_tet()
    f, fp = pair
    Np, mu, lam = 3, 0.7, 0.9
    topo = oracle_mod.topology(T)
    out, _, q, recv = oracle_mod.blocks_for_pairs(V, T, topo, np.array([mu]), lam, Np, np.array([0]), np.array([f]),
                                                  np.array([fp]))
    assert q[0] > 0
    mean, se = oracle_mod.mc_block(V, T, 0, f, fp, int(recv[0]), mu, lam, Np, nsamp=4 * 10 ** 6, seed=7 + f)
    z = np.abs(out[0] - mean) / np.maximum(se, 1e-12)
    assert z.max() < 5.0, (z.max(), np.unravel_index(z.argmax(), z.shape))


def test_monte_carlo_interior_neighbour_frame(oracle_mod):
    """A block received by the neighbour across an interior face uses the
    neighbour's face frame; MC checks that too."""
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    topo = oracle_mod.topology(m.tets)
    rows = np.nonzero(~topo.boundary)[0]
    r = int(rows[5])
    t, fp = divmod(r, 4)
    f = (fp + 1) % 4
    Np, mu = 2, 0.3
    out, _, _, recv = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, np.full(m.n_tets, mu), 0.5, Np,
                                                  np.array([t]), np.array([f]), np.array([fp]))
    assert int(recv[0]) != r and not topo.boundary[recv[0]]
    mean, se = oracle_mod.mc_block(m.verts, m.tets, t, f, fp, int(recv[0]), mu, 1.0, Np, nsamp=4 * 10 ** 6, seed=3)
    z = np.abs(out[0] - mean) / np.maximum(se, 1e-12)
    assert z.max() < 5.0


def test_conservation_weighted_column_sums(oracle_mod):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    Np = 3
    op = oracle_mod.assemble(m.verts, m.tets, np.zeros(m.n_tets), 1.0, Np, q=32)
    A = oracle_mod.face_areas(m.verts, m.tets)
    w = np.zeros((op.nrows, op.nb))
    w[:, 0] = np.sqrt(A)
    wB = oracle_mod.apply(op, w, trans=True)  # (B^T w)
    np.testing.assert_allclose(wB, w, atol=1e-11)
    # with damping the mass strictly decreases
    op2 = oracle_mod.assemble(m.verts, m.tets, np.full(m.n_tets, 0.5), 0.9, Np, q=32)
    wB2 = oracle_mod.apply(op2, w, trans=True)
    assert np.all(wB2[:, 0] < w[:, 0])


def test_adaptive_order_reaches_tolerance(oracle_mod):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    topo = oracle_mod.topology(m.tets)
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    sel = np.arange(0, 12 * m.n_tets, 17)
    out, _, q, _ = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, np.full(m.n_tets, 0.05), 0.95, 4, t[sel],
                                               f[sel], fp[sel], rtol=1e-12)
    assert np.all(q > 0)


def _contour_view_factor_area(P, Q):
    """A_P F_{P->Q} between two triangles by Stokes' theorem (the contour-integral
    form of the view factor): (1/2 pi) |sum over edge pairs of
    Int Int ln|x - y| dx . dy|.  The shared edge uses Int_0^1 Int_0^1 ln(L|s - t|)
    = ln L - 3/2; the other pairs are integrated numerically (scipy)."""
    from scipy.integrate import dblquad

    total = 0.0
    for i in range(3):
        a0, a1 = P[i], P[(i + 1) % 3]
        for j in range(3):
            b0, b1 = Q[j], Q[(j + 1) % 3]
            da, db = a1 - a0, b1 - b0
            dot = float(da @ db)
            if np.allclose(a0, b1) and np.allclose(a1, b0) or np.allclose(a0, b0) and np.allclose(a1, b1):
                total += dot * (np.log(np.linalg.norm(da)) - 1.5)
                continue
            val, _ = dblquad(lambda t, s: np.log(np.linalg.norm(a0 + s * da - b0 - t * db)), 0, 1, 0, 1,
                             epsabs=1e-13, epsrel=1e-12)
            total += dot * val
    return abs(total) / (2 * np.pi)


def test_view_factors_by_contour_integrals(oracle_mod):
    """The (0,0) entries at mu = 0 are view factors: B_00 = F_{l->l'} sqrt(A_l / A_l'),
    checked on a jittered tet against the contour-integral form."""
    pytest.importorskip("scipy")
    V, T = _jittered_tet()
    op = oracle_mod.assemble(V, T, np.array([0.0]), 1.0, 1, q=32)
    A = oracle_mod.face_areas(V, T)
    face = lambda f: V[[T[0, (f + 1 + k) % 4] for k in range(3)]]  # noqa: E731
    for f in range(4):
        for k, fp in enumerate([g for g in range(4) if g != f]):
            F = _contour_view_factor_area(face(f), face(fp)) / A[f]
            assert op.blocks[f, k, 0, 0] == pytest.approx(F * np.sqrt(A[f] / A[fp]), rel=1e-8), (f, fp)


def test_reciprocity_and_conservation_at_order_20(oracle_mod):
    """The largest basis of the cuboid verification (Sec. 4.1, N_p = 20,
    231 functions) on one jittered tet with fully reflecting faces at mu = 0:
    the reciprocity relation ties every test function to every trial function,
    and w^T B = w^T (mass conservation, Sec. 2) constrains all 231 trial
    columns of the (0,0) test row."""
    V, T = _jittered_tet()
    Np = 20
    op = oracle_mod.assemble(V, T, np.array([0.0]), 1.0, Np, q=32)
    N = oracle_mod.zernike_invnorm(Np)
    sign = np.array([(-1) ** n for n, m in oracle_mod.zernike_nm(Np)])
    fps = {f: [k for k in range(4) if k != f] for f in range(4)}
    blk = lambda f, fp: op.blocks[f, fps[f].index(fp)]
    for f in range(4):
        for fp in range(4):
            if fp != f:
                lhs = blk(f, fp) / N[:, None]
                rhs = (blk(fp, f) / N[:, None]).T * np.outer(sign, sign)
                np.testing.assert_allclose(lhs, rhs, atol=1e-10)
    A = oracle_mod.face_areas(V, T)
    w = np.zeros((op.nrows, op.nb))
    w[:, 0] = np.sqrt(A)
    np.testing.assert_allclose(oracle_mod.apply(op, w, trans=True), w, atol=1e-9)
