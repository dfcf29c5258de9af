"""GPU parity of the kernels for bases above N_p = 8 (N_b = 55 .. 231, the
orders of the cuboid verification of Sec. 4.1) against the FP64 oracle,
through the C ABI: assembled blocks, forward and transposed applications,
the GMRES-IR solve, the directed boundary source and the interior density.

Tolerances: blocks within 1e-5 of each block's max-norm (the method's FP32
entry tolerance) against the oracle at a fixed Gauss order of 64 per region
(order 32 is off by up to 2e-4 at N_p = 20 on the widest regions); FP32 applications
sum up to 693 products per entry, so 1e-5 of max |y|; FP64 vectors 1e-12.
"""
import numpy as np
import pytest

from gpu_helpers import block_rel_err, need_gpu, to_oracle_layout
from paper_1608_04607_gb300.inputs import kuhn_cube_mesh, random_boundary_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    need_gpu()
    from paper_1608_04607_gb300 import dfm

    dfm.load()
    return dfm


@pytest.fixture(scope="module")
def cube2():
    return kuhn_cube_mesh(2, jitter=0.2, seed=11)


def _gpu_op_as_oracle(oracle_mod, op, mesh, nt, Np):
    blocks = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), nt)
    t, f, fp = oracle_mod.pair_list(nt)
    dest = mesh.recv()[4 * t + fp].reshape(4 * nt, 3).astype(np.int64)
    return oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(blocks), dest=dest)


@pytest.mark.parametrize("Np", [9, 12, 16, 20])
def test_wide_assembly_matches_oracle(D, oracle_mod, cube2, Np):
    m = cube2
    mu, refl = 0.3, 0.85
    mesh = D.Mesh(m.verts, m.tets, refl=refl)
    op = D.Operator(mesh, Np, mu=mu, precision=D.F32)
    assert op.nb == (Np + 1) * (Np + 2) // 2
    got = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), m.n_tets)
    # every pair of a tet touching the boundary and of an interior-most tet
    cen = m.verts[m.tets].mean(axis=1)
    inner = int(np.argmin(np.abs(cen - 0.5).max(axis=1)))
    tsel = np.array([0, inner, m.n_tets - 1])
    topo = oracle_mod.topology(m.tets)
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    sel = np.isin(t, tsel)
    ref, _, _, _ = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, np.full(m.n_tets, mu), refl, Np, t[sel],
                                               f[sel], fp[sel], q=64)
    mine = got.reshape(-1, op.nb, op.nb)[sel]
    err = block_rel_err(mine, ref)
    assert err.max() <= 1e-5, err.max()
    # nodes were counted, and the blocks of the other tets are finite and non-zero
    assert D.op_nodes(op) > 0
    allb = got.reshape(-1, op.nb * op.nb)
    assert np.all(np.isfinite(allb)) and np.all(np.abs(allb).max(axis=1) > 0)


def test_wide_assembly_damping_moment(D, oracle_mod, cube2):
    """d B / d mu (moment 1) at N_p = 12 against the oracle's derivative blocks."""
    m = cube2
    Np, mu = 12, 0.2
    mesh = D.Mesh(m.verts, m.tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=mu, precision=D.F32, moment=1)
    got = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), m.n_tets).reshape(-1, op.nb, op.nb)
    topo = oracle_mod.topology(m.tets)
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    sel = np.isin(t, [5, 17])
    _, dref, _, _ = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, np.full(m.n_tets, mu), 0.9, Np, t[sel],
                                                f[sel], fp[sel], q=64, with_derivative=True)
    err = block_rel_err(got[sel], dref)
    assert err.max() <= 1e-5, err.max()


def test_wide_parameters_rejected(D, cube2):
    m = cube2
    mesh = D.Mesh(m.verts, m.tets, refl=0.9)
    for kw in (dict(Np=21), dict(Np=10, precision=D.BF16), dict(Np=10, precision=D.F64)):
        with pytest.raises(D.DFMError):
            D.Operator(mesh, kw["Np"], mu=0.1, precision=kw.get("precision", D.F32))
    op = D.Operator(mesh, 10, mu=0.1, precision=D.F32)
    import torch

    x = torch.zeros((op.n_rows, op.nb), dtype=torch.float32, device="cuda")
    with pytest.raises(D.DFMError) as e:
        op.precond(x, degree=4, precision=D.F16)
    assert e.value.code == D.DFM_ERR_UNSUPPORTED
    # the context is still usable
    y = op.apply(x)
    assert float(y.abs().max()) == 0.0


@pytest.mark.parametrize("Np", [12, 20])
@pytest.mark.parametrize("xdt", ["f64", "f32"])
def test_wide_apply_forward_and_transpose(D, oracle_mod, cube2, Np, xdt):
    import torch

    m = cube2
    mesh = D.Mesh(m.verts, m.tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=0.2, precision=D.F32)
    ref_op = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    rng = np.random.default_rng(Np)
    R = 2
    dt = torch.float64 if xdt == "f64" else torch.float32
    xt = torch.tensor(rng.standard_normal((R, m.n_rows, op.nb)), dtype=dt, device="cuda")
    x0t = torch.tensor(rng.standard_normal((R, m.n_rows, op.nb)), dtype=dt, device="cuda")
    tol = 1e-12 if xdt == "f64" else 1e-5
    for trans in (False, True):
        y = op.apply(xt, x0=x0t, alpha=-0.7, trans=trans).cpu().numpy()
        for r in range(R):
            yr = oracle_mod.apply(ref_op, xt[r].double().cpu().numpy(), trans=trans,
                                  x0=x0t[r].double().cpu().numpy(), alpha=-0.7)
            assert np.abs(y[r] - yr).max() <= tol * np.abs(yr).max()
        y2 = op.apply(xt[1].contiguous(), trans=trans).cpu().numpy()
        yr = oracle_mod.apply(ref_op, xt[1].double().cpu().numpy(), trans=trans)
        assert np.abs(y2 - yr).max() <= tol * np.abs(yr).max()


@pytest.mark.parametrize("Np,n", [(20, 1), (12, 2)])
def test_wide_solve_matches_same_operator(D, oracle_mod, Np, n):
    """GMRES-IR (FP32 Krylov, FP64 residual) against an FP64 solve of the same
    assembled blocks: dense LU on the single cube (24 rows x 231), the
    oracle's restarted GMRES to 1e-13 on the 48-tet cube."""
    m = kuhn_cube_mesh(n, jitter=0.2, seed=8)
    mesh = D.Mesh(m.verts, m.tets, refl=0.95)
    op = D.Operator(mesh, Np, mu=0.2, precision=D.F32)
    rows = random_boundary_rows(m, 2, seed=3)
    rho0 = D.source(mesh, Np, rows)
    rho, info = op.solve(rho0, tol=1e-10)
    assert info.resid <= 1e-10
    same = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    for r in range(len(rows)):
        b = rho0[r].cpu().numpy()
        ref = (oracle_mod.solve_dense(same, b) if n == 1
               else oracle_mod.solve_gmres(same, b, tol=1e-13, restart=100)[0])
        got = rho[r].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
        assert oracle_mod.residual(same, got, b) <= 1.5e-10


@pytest.mark.parametrize("Np", [12, 20])
def test_wide_source_directed_matches_oracle(D, oracle_mod, Np):
    m = kuhn_cube_mesh(3, jitter=0.2, seed=0)
    mesh = D.Mesh(m.verts, m.tets, refl=0.9)
    rows = random_boundary_rows(m, 11, seed=2)
    e1, e2, nn = oracle_mod.face_frames(m.verts, m.tets)
    rng = np.random.default_rng(Np)
    th = rng.uniform(0.0, 1.4, rows.size)
    ph = rng.uniform(0.0, 2 * np.pi, rows.size)
    dirs = (np.cos(th)[:, None] * nn[rows]
            + np.sin(th)[:, None] * (np.cos(ph)[:, None] * e1[rows] + np.sin(ph)[:, None] * e2[rows]))
    got = D.source_directed(mesh, Np, rows, dirs).cpu().numpy()
    ref = oracle_mod.source_directed(m.verts, m.tets, rows, Np, dirs=dirs)
    assert got.shape == ref.shape
    # the oracle's factorial closed form sums alternating terms of up to ~1e5
    # at n = 20, so near |p| = 1 it holds ~1e-10 (its order-20 pin: 2e-9)
    tol = 1e-12 if Np <= 12 else 2e-9
    np.testing.assert_allclose(got, ref, rtol=0, atol=tol * np.abs(ref).max())
    u = np.unique(rows)
    got = D.source_directed(mesh, Np, u, combine=True).cpu().numpy()
    ref = oracle_mod.source_directed(m.verts, m.tets, u, Np, combine=True)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_wide_interior_density_matches_oracle(D, oracle_mod):
    """The default split polar rule (24 points per direction) at N_p = 20 on
    the thin tets of the 768-tet cuboid against the oracle's restatement of
    the same rule (itself pinned against adaptive cubature), and at N_p = 12
    against the adaptive cubature of Eq. IntDens directly; the flat rule of
    order 32 against the oracle's flat rule of that order."""
    import torch

    from paper_1608_04607_gb300.inputs import kuhn_cuboid_mesh

    m = kuhn_cuboid_mesh(4)
    mesh = D.Mesh(m.verts, m.tets, refl=1.0)
    mu = 0.4 * np.pi
    tets = np.array([296, 343, 0, 511])
    cen = m.verts[m.tets].mean(axis=1)
    for Np in (12, 20):
        g, dg = D.interior_density(mesh, Np, tets, mu=mu, dgvec=torch.zeros((m.n_rows, (Np + 1) * (Np + 2) // 2),
                                                                              dtype=torch.float64, device="cuda"))
        g = g.cpu().numpy()
        dg = dg.cpu().numpy()
        for t in tets:
            gt = g[4 * t:4 * t + 4]
            gs = oracle_mod.interior_g_split(m.verts, m.tets, t, cen[t], mu, Np, n=24)
            assert np.abs(gt - gs).max() <= 1e-10 * np.abs(gs).max()
            if Np == 12 and t in (296, 0):
                ga, dga = oracle_mod.interior_g(m.verts, m.tets, t, cen[t], mu, Np, nq=None)
                assert np.abs(gt - ga).max() <= 1e-10 * np.abs(ga).max()
                assert np.abs(dg[4 * t:4 * t + 4] - dga).max() <= 1e-9 * np.abs(dga).max()
        # every other row is untouched
        others = np.setdiff1d(np.arange(m.n_tets), tets)
        assert np.all(g.reshape(m.n_tets, -1)[others] == 0.0)
    gf, _ = D.interior_density(mesh, 16, tets[:2], mu=mu, nq=32)
    gf = gf.cpu().numpy()
    for t in tets[:2]:
        go, _ = oracle_mod.interior_g(m.verts, m.tets, t, cen[t], mu, 16, nq=32)
        assert np.abs(gf[4 * t:4 * t + 4] - go).max() <= 1e-11 * np.abs(go).max()
