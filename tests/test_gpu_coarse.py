"""GPU tests of the two-level preconditioner (dfm_solve_opts.coarse): the
isotropic density on g^3 spatial aggregates solved exactly beside the
polynomial preconditioner on the e4m3 copy.  Solutions of the forward and the
transposed (adjoint) equation match an FP64 solve of the same assembled blocks
by the oracle's GMRES; batched solves ignore the option; g outside 0..4 is
refused."""
import numpy as np
import pytest

from gpu_helpers import need_gpu, to_oracle_layout
from paper_1608_04607_gb300.inputs import kuhn_cube_mesh, random_boundary_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    from paper_1608_04607_gb300 import dfm

    dfm.load()
    m = kuhn_cube_mesh(4, jitter=0.2, seed=8)
    mesh = dfm.Mesh(m.verts, m.tets, refl=0.95)
    Np = 3
    op = dfm.Operator(mesh, Np, mu=0.05, precision=dfm.F32)
    return dfm, m, mesh, op, Np


def _same(oracle_mod, op, mesh, m, Np):
    blocks = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), m.n_tets)
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    dest = mesh.recv()[4 * t + fp].reshape(4 * m.n_tets, 3).astype(np.int64)
    return oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(blocks), dest=dest)


@pytest.mark.parametrize("trans", [False, True])
def test_coarse_solve_matches_same_operator(setup, oracle_mod, trans):
    dfm, m, mesh, op, Np = setup
    rows = random_boundary_rows(m, 1, seed=4)
    rho0 = dfm.source(mesh, Np, rows)
    same = _same(oracle_mod, op, mesh, m, Np)
    ref = oracle_mod.solve_gmres(same, rho0[0].cpu().numpy(), tol=1e-13, restart=200, trans=trans)[0]
    its = {}
    for g in (0, 2, 3):
        rho, info = op.solve(rho0, tol=1e-10, precond_precision=dfm.FP8E4M3, transpose=trans, coarse=g)
        assert info.resid <= 1e-10
        got = rho[0].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref), g
        its[g] = info.iters
    # the coarse space's own applications are counted; the correction must not slow convergence much
    assert its[2] <= 1.2 * its[0] and its[3] <= 1.2 * its[0], its


def test_coarse_option_checks(setup, oracle_mod):
    dfm, m, mesh, op, Np = setup
    rows = random_boundary_rows(m, 2, seed=5)
    rho0 = dfm.source(mesh, Np, rows)
    with pytest.raises(dfm.DFMError) as e:
        op.solve(rho0[:1], tol=1e-8, precond_precision=dfm.FP8E4M3, coarse=5)
    assert e.value.code == dfm.DFM_ERR_ARG
    # batched: the option is ignored, the solutions stay right
    rho, info = op.solve(rho0, tol=1e-10, precond_precision=dfm.FP8E4M3, coarse=2)
    same = _same(oracle_mod, op, mesh, m, Np)
    for r in range(2):
        ref = oracle_mod.solve_gmres(same, rho0[r].cpu().numpy(), tol=1e-13, restart=200)[0]
        assert np.linalg.norm(rho[r].cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
