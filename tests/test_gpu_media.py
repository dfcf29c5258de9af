"""GPU parity of heterogeneous media (Sec. 3.3: the acoustic transmission law
across interfaces between tets of different speed c and fluid density rho_f,
Snell-scaled receiving momentum, and the specular reflection of the rest)
against the oracle's assemble_media: both parts of the operator block by
block, the application and the solve on the GPU's own blocks, and the adjoint
gradient with both parts' damping derivatives.

Two media fields on a jittered 2^3 Kuhn cube (48 tets):
 - impedance only (c = 1, rho_f varies): lambda_t = 4 z_i z_j / (z_i + z_j)^2
   is the same for every direction, the integrands stay smooth, and both parts'
   FP32 blocks meet the uniform medium's entry tolerance (1e-5 of each block's
   max);
 - speed and density vary: through a face into a slower or equally fast
   neighbour (c_i / c_j <= 1) the transmission law has no critical angle; the
   transmitted blocks meet 1e-5, the reflected ones, whose share
   ((z_i cos_r - z_j cos_t) / (z_i cos_r + z_j cos_t))^2 swings from 1 to
   its normal value within cos_r ~ sqrt(1 - (c_i/c_j)^2) of grazing, meet
   5e-3 with the default rule (order N_p + 6 per 60-degree patch) and 1e-5
   with order 24 on 30-degree patches in FP64 arithmetic (FP32 sums over
   that many nodes lose ~1e-5 of their own); into a faster neighbour lambda_t falls
   to zero at the critical angle with a square-root edge inside a direction
   region, where the oracle's adaptive rule does not reach its tolerance by
   its highest order (q_used < 0), so those blocks have no converged reference
   and are not compared.
Where no interface separates a face pair the reflected blocks are exactly 0."""
import numpy as np
import pytest

from gpu_helpers import block_rel_err, need_gpu, to_oracle_layout
from paper_1608_04607_gb300.inputs import kuhn_cube_mesh

pytestmark = pytest.mark.gpu

REFL = 0.8


@pytest.fixture(scope="module")
def D():
    need_gpu()
    from paper_1608_04607_gb300 import dfm

    dfm.load()
    return dfm


def _media(kind, nt):
    rng = np.random.default_rng(21)
    rhof = rng.uniform(0.5, 2.0, nt)
    c = np.ones(nt) if kind == "impedance" else rng.uniform(0.75, 1.3, nt)
    return c, rhof


def _gpu_oracle_op(oracle_mod, D, op, mesh, nt, Np, **kw):
    """The GPU's blocks (both parts) in the oracle's column layout."""
    recv = mesh.recv()
    t, f, fp = oracle_mod.pair_list(nt)
    blocks = to_oracle_layout(op.blocks().double().cpu().numpy(), recv, nt)
    rblocks = to_oracle_layout(op.blocks_reflected().double().cpu().numpy(), np.arange(4 * nt), nt)
    return oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(blocks),
                               dest=recv[4 * t + fp].reshape(4 * nt, 3).astype(np.int64),
                               rblocks=np.ascontiguousarray(rblocks),
                               rdest=(4 * t + fp).reshape(4 * nt, 3).astype(np.int64), **kw)


@pytest.mark.parametrize("kind", ["impedance", "snell"])
@pytest.mark.parametrize("Np", [2, 4])
def test_media_blocks_match_oracle(D, oracle_mod, kind, Np):
    import torch

    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    nt = m.n_tets
    c, rhof = _media(kind, nt)
    mu = np.random.default_rng(3).uniform(0.1, 0.5, nt)
    mesh = D.Mesh(m.verts, m.tets, refl=REFL)
    mu_t = torch.tensor(mu, device="cuda")
    op = D.Operator(mesh, Np, mu=mu_t, precision=D.F32, c=c, rho_f=rhof)
    ref = oracle_mod.assemble_media(m.verts, m.tets, mu, c, rhof, REFL, Np, rtol=1e-11)
    got = _gpu_oracle_op(oracle_mod, D, op, mesh, nt, Np)
    t, f, fp = oracle_mod.pair_list(nt)
    recv = mesh.recv()
    ratio = c[recv[4 * t + fp] // 4] / c[t]  # c_i / c_j across the exit face
    keep = ratio <= 1.0
    assert np.all(ref.q_used[keep] > 0)  # converged references only
    if kind == "impedance":
        assert keep.all()
    err = block_rel_err(got.blocks.reshape(-1, *ref.blocks.shape[-2:])[keep],
                        ref.blocks.reshape(-1, *ref.blocks.shape[-2:])[keep])
    assert err.max() <= 1e-5, (err.max(), np.median(err))
    live = np.abs(ref.rblocks).reshape(4 * nt * 3, -1).max(axis=1) > 0
    assert live.sum() > 20  # interfaces exist
    assert np.all(got.rblocks.reshape(4 * nt * 3, -1)[~live] == 0.0)
    sel = live & keep

    def rerr_of(o):
        return block_rel_err(o.rblocks.reshape(-1, *ref.rblocks.shape[-2:])[sel],
                             ref.rblocks.reshape(-1, *ref.rblocks.shape[-2:])[sel])

    rerr = rerr_of(got)
    assert rerr.max() <= (1e-5 if kind == "impedance" else 5e-3), (rerr.max(), np.median(rerr))
    if kind == "snell":  # the reflected blocks converge to the reference with a finer rule
        fine = D.Operator(mesh, Np, mu=mu_t, precision=D.F64, c=c, rho_f=rhof, quad_order=24, max_patch_deg=30.0)
        rerr = rerr_of(_gpu_oracle_op(oracle_mod, D, fine, mesh, nt, Np))
        print("snell reflected, FP64 fine rule:", Np, rerr.max(), np.median(rerr))
        assert rerr.max() <= 1e-5, (rerr.max(), np.median(rerr))


def test_media_apply_solve_and_adjoint(D, oracle_mod):
    """The application (forward and transposed, FP64 vectors) and the solve
    against the oracle on the GPU's own blocks of both parts; the adjoint
    gradient against the oracle's gradient with its own blocks and derivative
    blocks of both parts (impedance-only media: smooth integrands)."""
    import torch

    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    nt = m.n_tets
    c, rhof = _media("impedance", nt)
    rng = np.random.default_rng(5)
    mu = rng.uniform(0.2, 0.6, nt)
    Np = 2
    mesh = D.Mesh(m.verts, m.tets, refl=REFL)
    mu_t = torch.tensor(mu, device="cuda")
    op = D.Operator(mesh, Np, mu=mu_t, precision=D.F32, c=c, rho_f=rhof)
    same = _gpu_oracle_op(oracle_mod, D, op, mesh, nt, Np)
    x = torch.tensor(rng.standard_normal((2, mesh.n_rows, op.nb)), device="cuda")
    for trans in (False, True):
        y = op.apply(x, x0=x, alpha=-0.5, trans=trans).cpu().numpy()
        for r in range(2):
            xr = x[r].cpu().numpy()
            want = oracle_mod.apply(same, xr, trans=trans, x0=xr, alpha=-0.5)
            assert np.abs(y[r] - want).max() <= 1e-12 * np.abs(want).max(), trans
    recv = mesh.recv()
    rows = np.nonzero(recv == np.arange(mesh.n_rows))[0][[0, 9]]
    rho0 = D.source(mesh, Np, rows)
    rho, info = op.solve(rho0, tol=1e-11)
    assert info.resid <= 1e-11
    M = np.eye(same.nrows * same.nb) - oracle_mod.dense(same)
    for r in range(2):
        want = np.linalg.solve(M, rho0[r].cpu().numpy().ravel())
        assert np.linalg.norm(rho[r].cpu().numpy().ravel() - want) <= 1e-8 * np.linalg.norm(want)
    # adjoint gradient of J = sum_r g . rho_r
    receiver = np.array([20, 21])
    g, dg = D.interior_density(mesh, Np, receiver, weights=0.5, mu=mu_t)
    lam, dj, _ = op.adjoint(rho, g, dg, tol=1e-12)
    full = oracle_mod.assemble_media(m.verts, m.tets, mu, c, rhof, REFL, Np, rtol=1e-11, with_derivative=True)
    gref, dgref = oracle_mod.receiver_functional(m.verts, m.tets, mu, Np, receiver, nq=None)
    lam_ref = np.linalg.solve(np.eye(full.nrows * full.nb) - oracle_mod.dense(full).T,
                              gref.reshape(-1)).reshape(gref.shape)
    for r in range(2):
        b = oracle_mod.source_vector(m.verts, m.tets, rows[r:r + 1], Np)
        rho_ref = oracle_mod.solve_dense(full, b)
        grad = oracle_mod.gradient(full, rho_ref, lam_ref, dgref, nt)
        got = dj[r].cpu().numpy()
        assert np.abs(got - grad).max() <= 2e-5 * np.abs(grad).max(), np.abs(got - grad).max() / np.abs(grad).max()


def test_equal_media_give_the_uniform_operator(D):
    """c and rho_f equal everywhere: no interface, the reflected part is zero
    and the first part equals the uniform-media assembly bit for bit."""
    import torch

    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    mesh = D.Mesh(m.verts, m.tets, refl=REFL)
    ones = np.full(m.n_tets, 1.7)
    a = D.Operator(mesh, 3, mu=0.3, precision=D.F32, c=ones, rho_f=ones)
    b = D.Operator(mesh, 3, mu=0.3, precision=D.F32)
    assert torch.equal(a.blocks(), b.blocks())
    assert float(a.blocks_reflected().abs().max()) == 0.0
    with pytest.raises(D.DFMError):
        b.blocks_reflected()
