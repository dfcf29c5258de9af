"""Block flexible GMRES (dfm_solve_opts.block): the right-hand sides of a
group share one Krylov space.  Against LU of the same FP32 operator (the
oracle's dense solve of the GPU's own blocks) for several group sizes,
forward and transposed, with the FP16 and e4m3 preconditioner copies; a zero
right-hand side inside a block (a Gram pivot of zero: its basis column stays
zero) gives a zero solution without disturbing the others; and on a larger
cube the block solve needs fewer operator passes than the lockstep solve of
the same sources."""
import numpy as np
import pytest

from gpu_helpers import need_gpu, to_oracle_layout
from paper_1608_04607_gb300.inputs import kuhn_cube_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    need_gpu()
    from paper_1608_04607_gb300 import dfm

    dfm.load()
    return dfm


@pytest.fixture(scope="module")
def mesh161():
    m = kuhn_cube_mesh(3, jitter=0.2, seed=8)
    return m.verts, np.ascontiguousarray(m.tets[:-1])


def _dense(oracle_mod, op, mesh, nt, Np):
    blocks = to_oracle_layout(op.blocks().double().cpu().numpy(), mesh.recv(), nt)
    t, f, fp = oracle_mod.pair_list(nt)
    dest = mesh.recv()[4 * t + fp].reshape(4 * nt, 3).astype(np.int64)
    ref = oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(blocks), dest=dest)
    return np.eye(ref.nrows * ref.nb) - oracle_mod.dense(ref)


@pytest.mark.parametrize("Np,R,trans,prec", [(4, 2, False, "e4m3"), (4, 5, False, "e4m3"), (4, 8, True, "e4m3"),
                                             (3, 8, False, "f16"), (8, 4, False, "e4m3"), (2, 16, False, "f16")])
def test_block_solve_matches_lu(D, oracle_mod, mesh161, Np, R, trans, prec):
    import torch

    verts, tets = mesh161
    nt = tets.shape[0]
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=0.2, precision=D.F32)
    rng = np.random.default_rng(Np * 100 + R)
    b = torch.tensor(rng.standard_normal((R, 4 * nt, op.nb)), dtype=torch.float64, device="cuda")
    pp = {"e4m3": D.FP8E4M3, "f16": D.F16}[prec]
    x, info = op.solve(b, tol=1e-10, transpose=trans, precond_precision=pp, poly_degree=8, restart=6, block=1)
    assert info.resid <= 1e-10
    M = _dense(oracle_mod, op, mesh, nt, Np)
    for r in range(R):
        want = np.linalg.solve(M.T if trans else M, b[r].cpu().numpy().ravel())
        assert np.linalg.norm(x[r].cpu().numpy().ravel() - want) <= 1e-8 * np.linalg.norm(want), r


def test_zero_right_hand_side_in_a_block(D, oracle_mod, mesh161):
    import torch

    verts, tets = mesh161
    nt = tets.shape[0]
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, 4, mu=0.2, precision=D.F32)
    rng = np.random.default_rng(4)
    b = torch.tensor(rng.standard_normal((4, 4 * nt, op.nb)), dtype=torch.float64, device="cuda")
    b[2] = 0.0
    x, info = op.solve(b, tol=1e-10, precond_precision=D.FP8E4M3, poly_degree=8, restart=6, block=1)
    assert info.resid <= 1e-10
    assert float(x[2].abs().max()) == 0.0
    M = _dense(oracle_mod, op, mesh, nt, 4)
    for r in (0, 1, 3):
        want = np.linalg.solve(M, b[r].cpu().numpy().ravel())
        assert np.linalg.norm(x[r].cpu().numpy().ravel() - want) <= 1e-8 * np.linalg.norm(want)


def test_block_solve_needs_fewer_passes(D):
    """8 boundary sources on a jittered 10^3 cube (6,000 tets, N_p = 4, mu =
    0.05, reflection 0.95): the block space reaches 1e-8 in fewer operator
    passes than 8 lockstep Krylov spaces, and both agree to the tolerance."""
    import torch

    m = kuhn_cube_mesh(10, jitter=0.2, seed=1)
    mesh = D.Mesh(m.verts, m.tets, refl=0.95)
    op = D.Operator(mesh, 4, mu=0.05, precision=D.F32)
    recv = mesh.recv()
    bnd = np.nonzero(recv == np.arange(mesh.n_rows))[0]
    rows = np.random.default_rng(2).choice(bnd, 8, replace=False)
    b = D.source(mesh, 4, rows)
    kw = dict(tol=1e-8, precond_precision=D.FP8E4M3, poly_degree=32, restart=32)
    x_lock, i_lock = op.solve(b, block=0, **kw)
    x_blk, i_blk = op.solve(b, block=1, **kw)
    assert i_blk.resid <= 1e-8 and i_lock.resid <= 1e-8
    assert i_blk.iters < i_lock.iters, (i_blk.iters, i_lock.iters)
    d = (x_blk - x_lock).reshape(8, -1).norm(dim=1) / x_lock.reshape(8, -1).norm(dim=1)
    assert float(d.max()) <= 1e-7
