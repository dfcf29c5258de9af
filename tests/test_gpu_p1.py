"""GPU parity of the linear spatial basis (DFM_BASIS(Np, 1): three orthonormal
affine functions per face, the finer spatial approximation of Sec. 3.1 and
the end of Sec. 4.1) against the FP64 oracle, through the C ABI: assembled
blocks, applications, solves (unpreconditioned and with the e4m3
preconditioner copy), sources and the interior density.

The GPU integrates the spatial factor in closed form on the visible triangle
OBC of Sec. 3.3 (moments of the damping against the barycentric products); the
oracle clips the projected destination face and integrates the products of
the two spatial functions with a Gauss rule, so the routes share nothing.
Tolerances as for the constant basis: blocks within 1e-5 of each block's
max-norm against the oracle at Gauss order 64.
"""
import numpy as np
import pytest

from gpu_helpers import block_rel_err, need_gpu, to_oracle_layout
from paper_1608_04607_gb300.inputs import cuboid_rows_x0, kuhn_cube_mesh, kuhn_cuboid_mesh, random_boundary_rows

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
    return oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(blocks), dest=dest, ns=3)


@pytest.mark.parametrize("Np", [0, 2, 4, 8])
def test_p1_assembly_matches_oracle(D, oracle_mod, cube2, Np):
    m = cube2
    mu, refl = 0.3, 0.85
    mesh = D.Mesh(m.verts, m.tets, refl=refl)
    op = D.Operator(mesh, D.basis(Np, 1), mu=mu, precision=D.F32)
    nz = (Np + 1) * (Np + 2) // 2
    assert op.nb == 3 * nz and op.Np == D.basis(Np, 1)
    got = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), m.n_tets).reshape(-1, op.nb, op.nb)
    cen = m.verts[m.tets].mean(axis=1)
    inner = int(np.argmin(np.abs(cen - 0.5).max(axis=1)))
    topo = oracle_mod.topology(m.tets)
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    sel = np.isin(t, [0, inner, m.n_tets - 1])
    ref, _, _, _ = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, np.full(m.n_tets, mu), refl, Np, t[sel], f[sel],
                                               fp[sel], q=64, spatial=1)
    err = block_rel_err(got[sel], ref)
    assert err.max() <= 1e-5, err.max()
    # the constant functions' blocks are the piecewise-constant operator
    op0 = D.Operator(mesh, Np, mu=mu, precision=D.F32)
    b0 = to_oracle_layout(op0.blocks().cpu().numpy(), mesh.recv(), m.n_tets).reshape(-1, nz, nz)
    assert block_rel_err(got[:, :nz, :nz], b0).max() <= 5e-6


def test_p1_parameters_rejected(D, cube2):
    m = cube2
    mesh = D.Mesh(m.verts, m.tets, refl=0.9)
    for code, prec, kw in ((D.basis(9, 1), D.F32, {}), (D.basis(4, 1), D.BF16, {}), (D.basis(4, 1), D.F64, {}),
                           (D.basis(4, 2), D.F32, {}), (D.basis(4, 1), D.F32, {"moment": 1}),
                           (D.basis(4, 1), D.F32, {"c": np.ones(m.n_tets)})):
        with pytest.raises(D.DFMError):
            D.Operator(mesh, code, mu=0.1, precision=prec, **kw)
    import torch

    op = D.Operator(mesh, D.basis(2, 1), mu=0.1, precision=D.F32)
    x = torch.zeros((op.n_rows, op.nb), dtype=torch.float32, device="cuda")
    with pytest.raises(D.DFMError) as e:
        op.precond(x, degree=4, precision=D.F16)  # 18 unknowns per row: no preconditioner copy
    assert e.value.code == D.DFM_ERR_UNSUPPORTED
    assert float(op.apply(x).abs().max()) == 0.0  # the context is still usable


@pytest.mark.parametrize("Np", [0, 2, 4])
@pytest.mark.parametrize("xdt", ["f64", "f32"])
def test_p1_apply_forward_and_transpose(D, oracle_mod, cube2, Np, xdt):
    import torch

    m = cube2
    mesh = D.Mesh(m.verts, m.tets, refl=0.9)
    op = D.Operator(mesh, D.basis(Np, 1), mu=0.2, precision=D.F32)
    ref_op = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    rng = np.random.default_rng(Np + 1)
    dt = torch.float64 if xdt == "f64" else torch.float32
    xt = torch.tensor(rng.standard_normal((2, m.n_rows, op.nb)), dtype=dt, device="cuda")
    x0t = torch.tensor(rng.standard_normal((2, m.n_rows, op.nb)), dtype=dt, device="cuda")
    tol = 1e-12 if xdt == "f64" else 5e-6
    for trans in (False, True):
        y = op.apply(xt, x0=x0t, alpha=-0.7, trans=trans).cpu().numpy()
        for r in range(2):
            yr = oracle_mod.apply(ref_op, xt[r].double().cpu().numpy(), trans=trans,
                                  x0=x0t[r].double().cpu().numpy(), alpha=-0.7)
            assert np.abs(y[r] - yr).max() <= tol * np.abs(yr).max()


@pytest.mark.parametrize("Np,n,prec", [(4, 1, 0), (2, 2, 0), (4, 2, "fp8")])
def test_p1_solve_matches_same_operator(D, oracle_mod, Np, n, prec):
    """GMRES-IR to an FP64 residual of 1e-10 against an FP64 solve of the same
    blocks (dense LU on the single cube, the oracle's GMRES on the 48-tet cube);
    45 unknowns per row (N_p = 4) also run with the e4m3 preconditioner copy."""
    m = kuhn_cube_mesh(n, jitter=0.2, seed=8)
    mesh = D.Mesh(m.verts, m.tets, refl=0.95)
    code = D.basis(Np, 1)
    op = D.Operator(mesh, code, mu=0.2, precision=D.F32)
    rows = random_boundary_rows(m, 2, seed=3)
    rho0 = D.source(mesh, code, rows)
    kw = {"precond_precision": D.FP8E4M3} if prec == "fp8" else {}
    rho, info = op.solve(rho0, tol=1e-10, **kw)
    assert info.resid <= 1e-10
    same = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    for r in range(len(rows)):
        b = rho0[r].cpu().numpy()
        np.testing.assert_allclose(b, oracle_mod.source_vector(m.verts, m.tets, [rows[r]], Np, spatial=1),
                                   rtol=1e-14, atol=0)
        ref = (oracle_mod.solve_dense(same, b) if n == 1
               else oracle_mod.solve_gmres(same, b, tol=1e-13, restart=100)[0])
        got = rho[r].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("Np", [3, 8, 12])
def test_p1_source_directed_matches_oracle(D, oracle_mod, Np):
    m = kuhn_cube_mesh(3, jitter=0.2, seed=0)
    mesh = D.Mesh(m.verts, m.tets, refl=0.9)
    rows = random_boundary_rows(m, 9, seed=2)
    e1, e2, nn = oracle_mod.face_frames(m.verts, m.tets)
    rng = np.random.default_rng(Np)
    th = rng.uniform(0.0, 1.3, rows.size)
    ph = rng.uniform(0.0, 2 * np.pi, rows.size)
    dirs = (np.cos(th)[:, None] * nn[rows]
            + np.sin(th)[:, None] * (np.cos(ph)[:, None] * e1[rows] + np.sin(ph)[:, None] * e2[rows]))
    if Np > 8:  # the linear spatial basis stops at N_p = 8
        with pytest.raises(D.DFMError):
            D.source_directed(mesh, D.basis(Np, 1), rows, dirs)
        return
    got = D.source_directed(mesh, D.basis(Np, 1), rows, dirs).cpu().numpy()
    ref = oracle_mod.source_directed(m.verts, m.tets, rows, Np, dirs=dirs, spatial=1)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    u = np.unique(rows)
    got = D.source_directed(mesh, D.basis(Np, 1), u, combine=True).cpu().numpy()
    ref = oracle_mod.source_directed(m.verts, m.tets, u, Np, combine=True, spatial=1)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_p1_interior_density_matches_oracle(D, oracle_mod):
    """The default split polar rule on thin tets of the 768-tet cuboid and the
    flat rule of order 32 against the oracle's adaptive cubature and flat rule
    of Eq. IntDens with the face functions in the integrand; the per-tet
    readout of a linear-basis density."""
    import torch

    m = kuhn_cuboid_mesh(4)
    mesh = D.Mesh(m.verts, m.tets, refl=1.0)
    mu, Np = 0.4 * np.pi, 4
    code = D.basis(Np, 1)
    nb = 3 * (Np + 1) * (Np + 2) // 2
    tets = np.array([296, 343, 0])
    cen = m.verts[m.tets].mean(axis=1)
    g, dg = D.interior_density(mesh, code, tets, mu=mu)
    g, dg = g.cpu().numpy(), dg.cpu().numpy()
    assert g.shape == (m.n_rows, nb)
    for t in tets:
        ga, dga = oracle_mod.interior_g(m.verts, m.tets, t, cen[t], mu, Np, nq=None, spatial=1)
        assert np.abs(g[4 * t:4 * t + 4] - ga).max() <= 1e-10 * np.abs(ga).max()
        assert np.abs(dg[4 * t:4 * t + 4] - dga).max() <= 1e-9 * np.abs(dga).max()
    gf, _ = D.interior_density(mesh, code, tets[:2], mu=mu, nq=32)
    gf = gf.cpu().numpy()
    for t in tets[:2]:
        go, _ = oracle_mod.interior_g(m.verts, m.tets, t, cen[t], mu, Np, nq=32, spatial=1)
        assert np.abs(gf[4 * t:4 * t + 4] - go).max() <= 1e-11 * np.abs(go).max()
    # per-tet readout with the 3 nb unknowns per row
    rng = np.random.default_rng(5)
    rho = rng.standard_normal((m.n_rows, nb))
    dens = D.tet_density(mesh, code, torch.tensor(g, device="cuda"), torch.tensor(rho, device="cuda")).cpu().numpy()
    host = np.einsum("tk,tk->t", g.reshape(m.n_tets, -1), rho.reshape(m.n_tets, -1))
    np.testing.assert_allclose(dens, host, rtol=1e-12, atol=1e-12 * np.abs(host).max())


def test_p1_cuboid_matches_oracle(D, oracle_mod):
    """End to end on the 96-tet cuboid of Sec. 4.1 (normal-incidence beam,
    r = 1, mu = 0.4 pi) at N_p = 4 with the linear spatial basis: assembly,
    directed source, GMRES-IR and the per-tet readout (flat rule of order 32 on
    both sides) against the oracle's solve of its own operator.  The densities
    agree to the FP32 entry tolerance amplified by the conditioning; both give
    a larger mean error against Eq. ExactSol than the constant basis here (the
    linear functions do not reduce the angular smearing that dominates)."""
    m = kuhn_cuboid_mesh(2)
    mesh = D.Mesh(m.verts, m.tets, refl=1.0)
    mu, Np = 0.4 * np.pi, 4
    code = D.basis(Np, 1)
    op = D.Operator(mesh, code, mu=mu, precision=D.F32)
    rows = cuboid_rows_x0(m)
    rho0 = D.source_directed(mesh, code, rows, combine=True)
    rho, info = op.solve(rho0, tol=1e-10)
    g, _ = D.interior_density(mesh, code, np.arange(m.n_tets), mu=mu, nq=32)
    dens = D.tet_density(mesh, code, g, rho).cpu().numpy()
    ref_op = oracle_mod.assemble(m.verts, m.tets, np.full(m.n_tets, mu), 1.0, Np, q=32, spatial=1)
    ref_rho0 = oracle_mod.source_directed(m.verts, m.tets, rows, Np, combine=True, spatial=1)
    np.testing.assert_allclose(rho0.cpu().numpy(), ref_rho0, rtol=0, atol=1e-12 * np.abs(ref_rho0).max())
    ref_rho, _ = oracle_mod.solve_gmres(ref_op, ref_rho0, tol=1e-11, restart=200)
    ref = oracle_mod.tet_density(m.verts, m.tets, np.full(m.n_tets, mu), Np, ref_rho, nq=32, spatial=1)
    assert np.abs(dens - ref).max() <= 1e-3 * np.abs(ref).max(), np.abs(dens - ref).max() / np.abs(ref).max()
