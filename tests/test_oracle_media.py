"""Pins for the oracle's heterogeneous-media operator (Sec. 3.3 transmission
law with Snell's law, Sec. 3.2 Eq. B4DInt):

- the transmission probability: 4 z1 z2 / (z1 + z2)^2 at normal incidence,
  1 between equal media, 0 at grazing incidence and beyond the critical
  angle, 0 <= lambda_t <= 1, the same value for the reversed ray, and one
  minus the square of the textbook pressure reflection coefficient
  (Z2 cos th_i - Z1 cos th_t) / (Z2 cos th_i + Z1 cos th_t), Z1 the medium the
  ray leaves;
- equal media everywhere (c, rho_f not 1) give exactly the uniform operator
  and no reflected part;
- equal speeds with unequal impedances make lambda_t a constant per face:
  the transmitted blocks are that constant times the uniform blocks, the
  reflected blocks one minus it times the blocks of a specular wall;
- with mu = 0 and r = 1 the weighted column sums stay 1 (the transmitted
  and reflected parts of every ray add up to the ray, Sec. 2 conservation);
- Monte Carlo ray tracing of a transmitted and a reflected block across an
  interface with unequal speeds and impedances (Snell-bent directions).
"""
import dataclasses

import numpy as np
import pytest

from paper_1608_04607_gb300.inputs import kuhn_cube_mesh


def test_transmission_law(oracle_mod):
    T = oracle_mod.transmission
    assert T(1.0, 1.0, 2.0, 2.0) == pytest.approx(1.0, abs=1e-15)
    assert T(1.0, 1.7, 1.0, 3.0) == pytest.approx(4 * 3 / 16, abs=1e-15)  # normal incidence: no bending
    assert T(0.6, 1.0, 1.3, 1.3) == pytest.approx(1.0, abs=1e-15)
    assert T(1e-12, 0.8, 1.0, 2.0) < 1e-10  # grazing
    assert T(0.8, 2.0, 1.0, 1.0) == 0.0  # sin(theta_t) = 2 * 0.6 > 1: total internal reflection
    rng = np.random.default_rng(3)
    for _ in range(200):
        cr, k = rng.uniform(0.05, 1.0), rng.uniform(0.3, 3.0)
        zs, zd = rng.uniform(0.2, 5.0, 2)
        lt = T(cr, k, zs, zd)
        assert 0.0 <= lt <= 1.0
        s_t = k * np.sqrt(1 - cr * cr)
        if s_t < 1:  # textbook: 1 - r_p^2, r_p = (Z2 cos th_i - Z1 cos th_t) / (Z2 cos th_i + Z1 cos th_t)
            ct = np.sqrt(1 - s_t * s_t)
            assert lt == pytest.approx(1 - ((zd * cr - zs * ct) / (zd * cr + zs * ct)) ** 2, rel=1e-12)
        if s_t < 1:  # the reversed ray leaves the other medium at theta_t and arrives at theta_r
            assert T(np.sqrt(1 - s_t * s_t), 1.0 / k, zd, zs) == pytest.approx(lt, rel=1e-12)


def _mesh():
    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    return m.verts, m.tets


def test_equal_media_are_the_uniform_operator(oracle_mod):
    V, T = _mesh()
    nt = T.shape[0]
    mu = np.full(nt, 0.4)
    a = oracle_mod.assemble(V, T, mu, 0.9, 2, q=16)
    b = oracle_mod.assemble_media(V, T, mu, 1.7, 0.6, 0.9, 2, q=16)
    s = np.abs(a.blocks).max()
    assert np.abs(a.blocks - b.blocks).max() <= 1e-14 * s
    assert np.abs(b.rblocks).max() <= 1e-14 * s
    assert np.array_equal(a.dest, b.dest)


def test_impedance_mismatch_scales_blocks(oracle_mod):
    V, T = _mesh()
    nt = T.shape[0]
    rng = np.random.default_rng(5)
    rhof = rng.uniform(0.5, 2.0, nt)
    c = 1.3
    mu = np.full(nt, 0.3)
    Np = 2
    op = oracle_mod.assemble_media(V, T, mu, c, rhof, 0.8, Np, q=16)
    uni = oracle_mod.assemble(V, T, mu, 0.8, Np, q=16)
    topo = oracle_mod.topology(T)
    # every face a specular wall with r = 1: the reflection blocks of the exit face
    wall = dataclasses.replace(topo, recv=np.arange(4 * nt), boundary=np.ones(4 * nt, dtype=bool))
    t, f, fp = oracle_mod.pair_list(nt)
    refl, _, _, _ = oracle_mod.blocks_for_pairs(V, T, wall, mu, 1.0, Np, t, f, fp, q=16)
    refl = refl.reshape(4 * nt, 3, op.nb, op.nb)
    recv = topo.recv[4 * t + fp].reshape(4 * nt, 3)
    interior = ~topo.boundary[recv]
    z = c * rhof
    zs, zd = z[t].reshape(4 * nt, 3), z[recv // 4]
    lt = 4 * zs * zd / (zs + zd) ** 2
    s = np.abs(uni.blocks).max()
    want_t = np.where(interior[..., None, None], lt[..., None, None] * uni.blocks, uni.blocks)
    want_r = np.where(interior[..., None, None], (1 - lt)[..., None, None] * refl, 0.0)
    assert np.abs(op.blocks - want_t).max() <= 1e-13 * s
    assert np.abs(op.rblocks - want_r).max() <= 1e-13 * s
    assert np.array_equal(op.rdest.reshape(-1), 4 * t + fp)


def test_conservation_with_unequal_media(oracle_mod):
    V, T = _mesh()
    nt = T.shape[0]
    rng = np.random.default_rng(9)
    c = rng.uniform(0.6, 1.6, nt)
    rhof = rng.uniform(0.5, 2.0, nt)
    op = oracle_mod.assemble_media(V, T, np.zeros(nt), c, rhof, 1.0, 2, q=32)
    A = oracle_mod.face_areas(V, T)
    w = np.zeros((op.nrows, op.nb))
    w[:, 0] = np.sqrt(A)
    np.testing.assert_allclose(oracle_mod.apply(op, w, trans=True), w, atol=1e-11)
    # the dense form holds the same two parts
    M = oracle_mod.dense(op)
    np.testing.assert_allclose(M.T @ w.reshape(-1), w.reshape(-1), atol=1e-11)
    # some flux is reflected at interfaces and some is turned back by total internal reflection
    assert np.abs(op.rblocks).max() > 1e-3


@pytest.mark.parametrize("kind", [1, 2])
def test_monte_carlo_across_an_interface(oracle_mod, kind):
    V, T = _mesh()
    nt = T.shape[0]
    topo = oracle_mod.topology(T)
    r = int(np.nonzero(~topo.boundary)[0][5])
    t, fp = divmod(r, 4)
    f = (fp + 1) % 4
    i = int(topo.recv[r]) // 4
    c = np.ones(nt)
    rhof = np.ones(nt)
    c[i], rhof[i] = 0.7, 2.5  # slower, denser neighbour: bent towards the normal, no critical angle
    Np, mu = 2, 0.3
    op = oracle_mod.assemble_media(V, T, np.full(nt, mu), c, rhof, 0.5, Np)
    k = [g for g in range(4) if g != f].index(fp)
    J = 4 * t + f
    got = op.blocks[J, k] if kind == 1 else op.rblocks[J, k]
    row = int(op.dest[J, k]) if kind == 1 else r
    mean, se = oracle_mod.mc_block_media(V, T, t, f, fp, row, mu, kind, c[i] / c[t], c[t] * rhof[t],
                                         c[i] * rhof[i], Np, nsamp=4 * 10 ** 6, seed=11 + kind)
    z = np.abs(got - mean) / np.maximum(se, 1e-12)
    assert z.max() < 5.0, (z.max(), np.unravel_index(z.argmax(), z.shape))


def test_media_derivatives_match_differences(oracle_mod):
    V, T = _mesh()
    nt = T.shape[0]
    rng = np.random.default_rng(13)
    c = rng.uniform(0.8, 1.25, nt)
    rhof = rng.uniform(0.5, 2.0, nt)
    mu = np.full(nt, 0.4)
    op = oracle_mod.assemble_media(V, T, mu, c, rhof, 0.9, 2, q=16, with_derivative=True)
    h = 1e-5
    p = oracle_mod.assemble_media(V, T, mu + h, c, rhof, 0.9, 2, q=16)
    m = oracle_mod.assemble_media(V, T, mu - h, c, rhof, 0.9, 2, q=16)
    np.testing.assert_allclose(op.dblocks, (p.blocks - m.blocks) / (2 * h), atol=1e-9)
    np.testing.assert_allclose(op.drblocks, (p.rblocks - m.rblocks) / (2 * h), atol=1e-9)
    assert np.abs(op.drblocks).max() > 1e-4


def test_media_adjoint_gradient_matches_differences(oracle_mod):
    """dJ/dmu by the adjoint (transposed solve with both parts of B, and the
    derivative blocks of both) against central differences of J = g . rho."""
    V, T = _mesh()
    nt = T.shape[0]
    rng = np.random.default_rng(17)
    c = rng.uniform(0.8, 1.25, nt)
    rhof = rng.uniform(0.5, 2.0, nt)
    mu = rng.uniform(0.3, 0.6, nt)
    Np = 1
    topo = oracle_mod.topology(T)
    rows = np.nonzero(topo.boundary)[0][[0, 9]]
    b = oracle_mod.source_vector(V, T, rows, Np)
    g, dg = oracle_mod.receiver_functional(V, T, mu, Np, [20, 21])
    op = oracle_mod.assemble_media(V, T, mu, c, rhof, 0.8, Np, q=16, with_derivative=True)
    rho = oracle_mod.solve_dense(op, b)
    lam = np.linalg.solve(np.eye(op.nrows * op.nb) - oracle_mod.dense(op).T, g.reshape(-1)).reshape(g.shape)
    grad = oracle_mod.gradient(op, rho, lam, dg, nt)

    def J(mv):
        o = oracle_mod.assemble_media(V, T, mv, c, rhof, 0.8, Np, q=16)
        gv, _ = oracle_mod.receiver_functional(V, T, mv, Np, [20, 21])
        return float(np.sum(gv * oracle_mod.solve_dense(o, b)))

    h = 1e-5
    for e in (0, 20, 33):
        mp, mm = mu.copy(), mu.copy()
        mp[e] += h
        mm[e] -= h
        assert grad[e] == pytest.approx((J(mp) - J(mm)) / (2 * h), rel=1e-5, abs=1e-10)
