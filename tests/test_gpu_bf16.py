"""GPU parity of BF16 operator storage (the format of the 45-function,
64-source workload): assembly, application, the batched GMRES-IR solve and
the adjoint on a BF16 operator, against the oracle on the same BF16 blocks.

Reading of "solution <= 1e-6 after refinement" for a reduced-precision
operator: the solve is compared with an FP64 LU solve of the SAME assembled
operator (the GPU's BF16 blocks widened to FP64); the rounding of the blocks
themselves (relative 2^-9) is the operator error, checked against the FP32
assembly bit for bit."""
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
def small(D):
    m = kuhn_cube_mesh(2, jitter=0.2, seed=3)
    mesh = D.Mesh(m.verts, m.tets, refl=0.9)
    return m, mesh


def _as_oracle(oracle_mod, op, mesh, nt, Np, dblocks=None):
    blocks = to_oracle_layout(op.blocks().float().cpu().numpy(), mesh.recv(), nt)
    t, f, fp = oracle_mod.pair_list(nt)
    dest = mesh.recv()[4 * t + fp].reshape(4 * nt, 3).astype(np.int64)
    return oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(blocks), dest=dest, dblocks=dblocks)


@pytest.mark.parametrize("Np", [4, 8])
def test_bf16_assembly_is_the_rounded_fp32_assembly(D, small, Np):
    import torch

    m, mesh = small
    op32 = D.Operator(mesh, Np, mu=0.3, precision=D.F32)
    op16 = D.Operator(mesh, Np, mu=0.3, precision=D.BF16)
    assert op16.bytes * 2 == op32.bytes
    assert torch.equal(op32.blocks().to(torch.bfloat16), op16.blocks())


@pytest.mark.parametrize("xdt", ["f32", "f64"])
def test_bf16_apply_matches_oracle(D, oracle_mod, small, xdt):
    import torch

    m, mesh = small
    Np = 8
    op = D.Operator(mesh, Np, mu=0.3, precision=D.BF16)
    ref = _as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    rng = np.random.default_rng(2)
    dt = torch.float32 if xdt == "f32" else torch.float64
    x = torch.tensor(rng.standard_normal((2, mesh.n_rows, op.nb)), dtype=dt, device="cuda")
    x0 = torch.tensor(rng.standard_normal((2, mesh.n_rows, op.nb)), dtype=dt, device="cuda")
    tol = 2e-6 if xdt == "f32" else 1e-12
    for trans in (False, True):
        y = op.apply(x, x0=x0, alpha=-0.7, trans=trans).cpu().numpy()
        for r in range(2):
            yr = oracle_mod.apply(ref, x[r].double().cpu().numpy(), trans=trans, x0=x0[r].double().cpu().numpy(),
                                  alpha=-0.7)
            assert np.abs(y[r] - yr).max() <= tol * np.abs(yr).max()


@pytest.mark.parametrize("precond", [0, "fp8"])
def test_bf16_batched_solve_matches_lu(D, oracle_mod, small, precond):
    m, mesh = small
    Np = 8
    op = D.Operator(mesh, Np, mu=0.3, precision=D.BF16)
    ref = _as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    recv = mesh.recv()
    rows = np.nonzero(recv == np.arange(mesh.n_rows))[0][[0, 5, 11]]
    rho0 = D.source(mesh, Np, rows)
    pp = D.FP8E4M3 if precond == "fp8" else 0
    rho, info = op.solve(rho0, tol=1e-9, precond_precision=pp, restart=32)
    assert info.resid <= 1e-9
    M = np.eye(ref.nrows * ref.nb) - oracle_mod.dense(ref)
    got = rho.cpu().numpy()
    for r in range(len(rows)):
        want = np.linalg.solve(M, rho0[r].cpu().numpy().ravel())
        assert np.linalg.norm(got[r].ravel() - want) <= 1e-6 * np.linalg.norm(want)


def test_bf16_adjoint_matches_oracle_on_the_same_blocks(D, oracle_mod, small):
    """lambda from the transposed BF16 solve vs LU; dJ/dmu vs the oracle's
    gradient formula with the oracle's own dB/dmu and the BF16 operator's
    rho and lambda."""
    import torch

    m, mesh = small
    Np = 4
    rng = np.random.default_rng(9)
    mu = rng.uniform(0.2, 0.6, m.n_tets)
    mu_t = torch.tensor(mu, device="cuda")
    op = D.Operator(mesh, Np, mu=mu_t, precision=D.BF16)
    recv = mesh.recv()
    rows = np.nonzero(recv == np.arange(mesh.n_rows))[0][[1, 6]]
    rho0 = D.source(mesh, Np, rows)
    rho, _ = op.solve(rho0, tol=1e-12)
    receiver = np.array([20, 21, 30])
    g, dg = D.interior_density(mesh, Np, receiver, weights=1.0 / 3, mu=mu_t)
    lam, dj, _ = op.adjoint(rho, g, dg, tol=1e-12)
    full = oracle_mod.assemble(m.verts, m.tets, mu, 0.9, Np, rtol=1e-10, with_derivative=True)
    same = _as_oracle(oracle_mod, op, mesh, m.n_tets, Np, dblocks=full.dblocks)
    M = np.eye(same.nrows * same.nb) - oracle_mod.dense(same)
    lref = np.linalg.solve(M.T, g.cpu().numpy().ravel())
    assert np.linalg.norm(lam.cpu().numpy().ravel() - lref) <= 1e-9 * np.linalg.norm(lref)
    _, dgref = oracle_mod.receiver_functional(m.verts, m.tets, mu, Np, receiver, nq=None)
    for r in range(2):
        rref = np.linalg.solve(M, rho0[r].cpu().numpy().ravel()).reshape(same.nrows, same.nb)
        gref = oracle_mod.gradient(same, rref, lref.reshape(same.nrows, same.nb), dgref, m.n_tets)
        got = dj[r].cpu().numpy()
        assert np.abs(got - gref).max() <= 2e-5 * np.abs(gref).max()


@pytest.mark.parametrize("Np,R", [(8, 4), (8, 9), (8, 17), (4, 8), (3, 16)])
def test_bf16_apply_many_rhs_on_tensor_cores(D, oracle_mod, small, Np, R):
    """Four or more FP32 right-hand sides on a BF16 operator run on tensor
    cores (each coefficient split exactly into three BF16 parts, FP32
    accumulation): the same 2e-6 of max |y| as the CUDA-core application,
    with x0 given, aliasing x, or absent; R = 17 spans two launches (16 + 1)."""
    import torch

    m, mesh = small
    op = D.Operator(mesh, Np, mu=0.3, precision=D.BF16)
    ref = _as_oracle(oracle_mod, op, mesh, m.n_tets, Np)
    rng = np.random.default_rng(R)
    x = torch.tensor(rng.standard_normal((R, mesh.n_rows, op.nb)), dtype=torch.float32, device="cuda")
    x0 = torch.tensor(rng.standard_normal((R, mesh.n_rows, op.nb)), dtype=torch.float32, device="cuda")
    for kind in ("x0", "alias", "none"):
        xx0 = {"x0": x0, "alias": x, "none": None}[kind]
        y = op.apply(x, x0=xx0, alpha=-0.7).cpu().numpy()
        for r in range(R):
            base = None if xx0 is None else xx0[r].double().cpu().numpy()
            yr = oracle_mod.apply(ref, x[r].double().cpu().numpy(), x0=base, alpha=-0.7)
            assert np.abs(y[r] - yr).max() <= 2e-6 * np.abs(yr).max(), (kind, r)
