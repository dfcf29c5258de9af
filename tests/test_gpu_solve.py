"""GPU parity of the block-sparse operator application, sources and the
stationary solvers against the FP64 oracle, through the C ABI.

The solve is checked two ways (a solution error bound needs both):
 - against an FP64 solve of the SAME assembled operator (the GPU blocks
   widened to FP64 and solved by the oracle's dense LU), which isolates the
   solver: relative error <= 1e-6 after refinement (1e-9 for the FP64 path);
 - end to end against the oracle's own operator, where the quadrature error
   of the blocks (~3e-7) is amplified by the conditioning of I - B.
"""
import numpy as np
import pytest

from gpu_helpers import need_gpu, to_oracle_layout
from paper_1608_04607_gb300.inputs import kuhn_cube_mesh, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    need_gpu()
    from paper_1608_04607_gb300 import dfm

    dfm.load()
    return dfm


def _gpu_op_as_oracle(oracle_mod, op, mesh, nt, Np):
    blocks = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), nt)
    t, f, fp = oracle_mod.pair_list(nt)
    dest = mesh.recv()[4 * t + fp].reshape(4 * nt, 3).astype(np.int64)
    return oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(blocks), dest=dest)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("xdt", ["f64", "f32"])
def test_apply_forward_and_transpose(D, oracle_mod, prec, xdt):
    import torch

    m = kuhn_cube_mesh(3, jitter=0.2, seed=8)
    Np = 4
    mesh = D.Mesh(m.verts, m.tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=0.2, precision=prec)
    ref_op = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    rng = np.random.default_rng(1)
    R = 3
    x = rng.standard_normal((R, 4 * m.n_tets, op.nb))
    x0 = rng.standard_normal((R, 4 * m.n_tets, op.nb))
    dt = torch.float64 if xdt == "f64" else torch.float32
    xt = torch.tensor(x, dtype=dt, device="cuda")
    x0t = torch.tensor(x0, dtype=dt, device="cuda")
    tol = 1e-12 if (xdt == "f64") else 2e-6
    for trans in (False, True):
        y = op.apply(xt, x0=x0t, alpha=-0.7, trans=trans).cpu().numpy()
        for r in range(R):
            xr = xt[r].double().cpu().numpy()
            x0r = x0t[r].double().cpu().numpy()
            yr = oracle_mod.apply(ref_op, xr, trans=trans, x0=x0r, alpha=-0.7)
            assert np.abs(y[r] - yr).max() <= tol * np.abs(yr).max()
        # x0 = NULL
        y2 = op.apply(xt, alpha=1.0, trans=trans).cpu().numpy()
        yr = oracle_mod.apply(ref_op, xt[0].double().cpu().numpy(), trans=trans)
        assert np.abs(y2[0] - yr).max() <= tol * np.abs(yr).max()


@pytest.mark.parametrize("Np", [2, 4])
def test_apply_alternating_sweeps_bit_identical(D, oracle_mod, Np):
    """Consecutive applications sweep the operator rows in opposite
    directions; every output row is still formed in one fixed order, so
    repeated applications agree bit for bit.  The mesh drops one tet of the
    Kuhn cube (161 tets, 644 rows), so the last tile of both the forward
    (rows) and the transposed (source tets) pipeline is ragged."""
    import torch

    m = kuhn_cube_mesh(3, jitter=0.2, seed=8)
    tets = np.ascontiguousarray(m.tets[:-1])
    nt = tets.shape[0]
    mesh = D.Mesh(m.verts, tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=0.2, precision=1)
    ref_op = _gpu_op_as_oracle(oracle_mod, op, mesh, nt, Np)
    rng = np.random.default_rng(5)
    xt = torch.tensor(rng.standard_normal((2, 4 * nt, op.nb)), dtype=torch.float32, device="cuda")
    x0t = torch.tensor(rng.standard_normal((2, 4 * nt, op.nb)), dtype=torch.float32, device="cuda")
    for trans in (False, True):
        ys = [op.apply(xt, x0=x0t, alpha=-0.7, trans=trans).clone() for _ in range(3)]
        assert torch.equal(ys[0], ys[1]) and torch.equal(ys[1], ys[2])
        y = ys[0].cpu().numpy()
        for r in range(2):
            yr = oracle_mod.apply(ref_op, xt[r].double().cpu().numpy(), trans=trans,
                                  x0=x0t[r].double().cpu().numpy(), alpha=-0.7)
            assert np.abs(y[r] - yr).max() <= 2e-6 * np.abs(yr).max()


@pytest.mark.parametrize("R", [8, 16])
@pytest.mark.parametrize("xdt", ["f64", "f32"])
def test_apply_many_rhs_with_x0(D, oracle_mod, R, xdt):
    """Many right-hand sides with x0: the staged rows no longer fit eight per
    tile (FP64 vectors), so tiles shrink to 7 or 5 rows and the x0 slices of
    such tiles are read directly instead of by 16-byte bulk copies."""
    import torch

    m = kuhn_cube_mesh(3, jitter=0.2, seed=8)
    Np = 4
    mesh = D.Mesh(m.verts, m.tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=0.2, precision=1)
    ref_op = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    rng = np.random.default_rng(R)
    dt = torch.float64 if xdt == "f64" else torch.float32
    xt = torch.tensor(rng.standard_normal((R, 4 * m.n_tets, op.nb)), dtype=dt, device="cuda")
    x0t = torch.tensor(rng.standard_normal((R, 4 * m.n_tets, op.nb)), dtype=dt, device="cuda")
    y = op.apply(xt, x0=x0t, alpha=-0.7).cpu().numpy()
    tol = 1e-12 if xdt == "f64" else 2e-6
    for r in range(R):
        yr = oracle_mod.apply(ref_op, xt[r].double().cpu().numpy(), x0=x0t[r].double().cpu().numpy(), alpha=-0.7)
        assert np.abs(y[r] - yr).max() <= tol * np.abs(yr).max()


def test_source_vector(D, oracle_mod):
    m = kuhn_cube_mesh(3, jitter=0.2, seed=8)
    mesh = D.Mesh(m.verts, m.tets)
    rows = np.array([5, 77, 300, 5])
    got = D.source(mesh, 3, rows).cpu().numpy()
    for s, r in enumerate(rows):
        ref = oracle_mod.source_vector(m.verts, m.tets, [r], 3)
        np.testing.assert_allclose(got[s], ref, rtol=1e-15, atol=0)


def test_single_cube_neumann(D, oracle_mod):
    """The small single-cube workload: FP64 operator, Neumann series to 1e-10."""
    import torch

    w = workload("kuhn1_np2")
    m = w["mesh"]
    mesh = D.Mesh(m.verts, m.tets, refl=w["refl"])
    op = D.Operator(mesh, w["Np"], mu=0.1, precision=D.F64)
    rho0 = D.source(mesh, w["Np"], w["sources"])
    rho, info = op.solve(rho0, method=D.NEUMANN, tol=1e-10)
    assert info.iters > 10
    got = rho[0].cpu().numpy()
    same = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, w["Np"])
    ref_same = oracle_mod.solve_dense(same, rho0[0].cpu().numpy())
    # stopping on the increment |x_k+1 - x_k| <= tol |x_k+1| leaves an error of at
    # most about tol * r / (1 - r), r the spectral radius of B
    r = np.max(np.abs(np.linalg.eigvals(oracle_mod.dense(same))))
    bound = 1e-10 * r / (1 - r)
    assert np.linalg.norm(got - ref_same) <= 1.5 * bound * np.linalg.norm(ref_same)
    own = oracle_mod.assemble(m.verts, m.tets, w["mu"], w["refl"], w["Np"])
    ref_own = oracle_mod.solve_dense(own, oracle_mod.source_vector(m.verts, m.tets, w["sources"], w["Np"]))
    assert np.linalg.norm(got - ref_own) <= 1e-5 * np.linalg.norm(ref_own)
    # GMRES on the FP64 operator agrees
    rho2, info2 = op.solve(rho0, method=D.GMRES, tol=1e-12)
    assert np.linalg.norm(rho2[0].cpu().numpy() - ref_same) <= 1e-10 * np.linalg.norm(ref_same)


@pytest.mark.parametrize("method", ["ir", "gmres64"])
def test_gmres_jittered(D, oracle_mod, method):
    m = kuhn_cube_mesh(3, jitter=0.2, seed=8)
    Np = 3
    mesh = D.Mesh(m.verts, m.tets, refl=0.95)
    prec = D.F32 if method == "ir" else D.F64
    op = D.Operator(mesh, Np, mu=0.05, precision=prec)
    rows = [int(np.nonzero(mesh.recv() == np.arange(mesh.n_rows))[0][3])]
    rho0 = D.source(mesh, Np, rows)
    meth = D.GMRES_IR if method == "ir" else D.GMRES
    rho, info = op.solve(rho0, method=meth, tol=1e-10, restart=40)
    assert info.resid <= 1e-10
    same = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    b = rho0[0].cpu().numpy()
    ref = oracle_mod.solve_dense(same, b)
    got = rho[0].cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    # the library's FP64 residual agrees with the oracle's
    assert oracle_mod.residual(same, got, b) <= 1.5e-10


def test_solver_reports_nonconvergence(D):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=8)
    mesh = D.Mesh(m.verts, m.tets, refl=0.95)
    op = D.Operator(mesh, 2, mu=0.05, precision=D.F64)
    rho0 = D.source(mesh, 2, [0])
    with pytest.raises(D.DFMError) as e:
        op.solve(rho0, method=D.NEUMANN, tol=1e-14, max_iter=5)
    assert e.value.code == D.DFM_ERR_NOT_CONVERGED
    rho, info = op.solve(rho0, method=D.GMRES_IR if op.precision == D.F32 else D.GMRES, tol=1e-14, max_iter=3,
                         raise_on_nonconvergence=False)
    assert info.iters <= 4


@pytest.mark.parametrize("poly", [1, 4, 16])
def test_polynomial_preconditioning_and_transpose(D, oracle_mod, poly):
    """GMRES-IR with the Neumann-polynomial right preconditioner of degree d,
    forward and transposed (adjoint) systems, against LU on the same operator."""
    m = kuhn_cube_mesh(3, jitter=0.2, seed=9)
    Np = 2
    mesh = D.Mesh(m.verts, m.tets, refl=0.95)
    op = D.Operator(mesh, Np, mu=0.05, precision=D.F32)
    same = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    M = np.eye(same.nrows * same.nb) - oracle_mod.dense(same)
    rng = np.random.default_rng(poly)
    import torch

    b = torch.tensor(rng.standard_normal((1, mesh.n_rows, op.nb)), device="cuda")
    for trans in (False, True):
        x, info = op.solve(b, method=D.GMRES_IR, tol=1e-10, poly_degree=poly, transpose=trans)
        ref = np.linalg.solve(M.T if trans else M, b[0].cpu().numpy().ravel())
        got = x[0].cpu().numpy().ravel()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
        assert info.resid <= 1e-10


def test_apply_rejects_misaligned_vectors(D):
    """The operator application streams x through 16-byte bulk copies; a
    misaligned x is refused on the host before any launch."""
    import torch

    m = kuhn_cube_mesh(2, jitter=0.2, seed=8)
    mesh = D.Mesh(m.verts, m.tets)
    op = D.Operator(mesh, 2, mu=0.1)
    buf = torch.zeros(mesh.n_rows * op.nb + 1, dtype=torch.float32, device="cuda")
    x = buf[1:].view(mesh.n_rows, op.nb)
    with pytest.raises(D.DFMError) as e:
        op.apply(x)
    assert e.value.code == D.DFM_ERR_ARG


@pytest.mark.parametrize("R,batch", [(5, 0), (5, 2)])
def test_batched_refinement_matches_lu(D, oracle_mod, R, batch):
    """R right-hand sides iterated in lockstep (one operator pass per
    polynomial hop for all of them), in groups of `batch`, against LU."""
    import torch

    m = kuhn_cube_mesh(3, jitter=0.2, seed=10)
    Np = 2
    mesh = D.Mesh(m.verts, m.tets, refl=0.95)
    op = D.Operator(mesh, Np, mu=0.05, precision=D.F32)
    same = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    M = np.eye(same.nrows * same.nb) - oracle_mod.dense(same)
    rng = np.random.default_rng(R + batch)
    b = rng.standard_normal((R, mesh.n_rows, op.nb))
    b[2] *= 1e-3  # different scales converge at different steps
    bt = torch.tensor(b, device="cuda")
    x, info = op.solve(bt, method=D.GMRES_IR, tol=1e-10, batch=batch)
    assert info.resid <= 1e-10
    for r in range(R):
        ref = np.linalg.solve(M, b[r].ravel())
        got = x[r].cpu().numpy().ravel()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("R", [1, 3])
def test_flexible_gmres_with_16bit_preconditioner(D, oracle_mod, prec, R):
    """The polynomial preconditioner's hops run on a 16-bit copy of the blocks
    (flexible GMRES); the solution still meets the FP64 residual tolerance and
    equals LU on the FP32 operator."""
    import torch

    m = kuhn_cube_mesh(3, jitter=0.2, seed=13)
    Np = 2
    mesh = D.Mesh(m.verts, m.tets, refl=0.95)
    op = D.Operator(mesh, Np, mu=0.05, precision=D.F32)
    same = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    M = np.eye(same.nrows * same.nb) - oracle_mod.dense(same)
    rng = np.random.default_rng(R)
    b = rng.standard_normal((R, mesh.n_rows, op.nb))
    pp = D.F16 if prec == "f16" else D.BF16
    x, info = op.solve(torch.tensor(b, device="cuda"), method=D.GMRES_IR, tol=1e-10, precond_precision=pp)
    assert info.resid <= 1e-10
    for r in range(R):
        ref = np.linalg.solve(M, b[r].ravel())
        assert np.linalg.norm(x[r].cpu().numpy().ravel() - ref) <= 1e-8 * np.linalg.norm(ref)
    # re-assembly refreshes the 16-bit copy
    op.reassemble(0.2)
    x2, info2 = op.solve(torch.tensor(b, device="cuda"), method=D.GMRES_IR, tol=1e-10, precond_precision=pp)
    same2 = _gpu_op_as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    M2 = np.eye(same2.nrows * same2.nb) - oracle_mod.dense(same2)
    ref2 = np.linalg.solve(M2, b[0].ravel())
    assert np.linalg.norm(x2[0].cpu().numpy().ravel() - ref2) <= 1e-8 * np.linalg.norm(ref2)


def test_sampled_kernel_timing_counts_every_launch(D):
    """dfm_stats_enable(n) times every n-th launch of a kernel but reports all
    launches and scales the summed time to them."""
    import torch

    m = kuhn_cube_mesh(3, jitter=0.2, seed=8)
    mesh = D.Mesh(m.verts, m.tets, refl=0.9)
    op = D.Operator(mesh, 4, mu=0.2, precision=1)
    x = torch.randn((mesh.n_rows, op.nb), device="cuda", dtype=torch.float32)
    for every in (1, 4):
        D.stats_reset()
        D.stats_enable(every)
        for _ in range(10):
            op.apply(x, x0=x, alpha=-1.0)
        D.stats_enable(False)
        n, ms = D.kernel_stats(D.KERNEL_SPMV)
        assert n == 10 and ms > 0
    D.stats_reset()
