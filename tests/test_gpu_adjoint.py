"""GPU parity of the receiver functional (Eq. IntDens) and the adjoint
gradient dJ/dmu (fused lambda^T dB/dmu rho contraction) against the FP64
oracle, plus central finite differences of the GPU forward solve."""
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
def problem(D):
    import torch

    m = kuhn_cube_mesh(2, jitter=0.2, seed=11)
    rng = np.random.default_rng(5)
    mu = rng.uniform(0.2, 0.6, m.n_tets)
    Np = 2
    mesh = D.Mesh(m.verts, m.tets, refl=0.8)
    recv = mesh.recv()
    rows = np.nonzero(recv == np.arange(mesh.n_rows))[0][[0, 7]]
    receiver = np.array([20, 21, 30])
    return dict(m=m, mu=mu, Np=Np, mesh=mesh, rows=rows, receiver=receiver,
                mu_t=torch.tensor(mu, device="cuda"))


def test_interior_density_matches_oracle(D, oracle_mod, problem):
    p = problem
    m = p["m"]
    w = 1.0 / len(p["receiver"])
    g, dg = D.interior_density(p["mesh"], p["Np"], p["receiver"], weights=w, mu=p["mu_t"])
    # the default rule against the oracle's adaptive cubature (the definition)
    gref, dgref = oracle_mod.receiver_functional(m.verts, m.tets, p["mu"], p["Np"], p["receiver"], nq=None)
    np.testing.assert_allclose(g.cpu().numpy(), gref, rtol=0, atol=1e-10 * np.abs(gref).max())
    dgr = np.zeros_like(gref)
    for e, d in dgref.items():
        dgr[4 * e:4 * e + 4] = d
    np.testing.assert_allclose(dg.cpu().numpy(), dgr, rtol=0, atol=1e-10 * np.abs(dgr).max())


def test_adjoint_gradient_matches_oracle(D, oracle_mod, problem):
    import torch

    p = problem
    m = p["m"]
    mesh = p["mesh"]
    op = D.Operator(mesh, p["Np"], mu=p["mu_t"], precision=D.F32)
    rho0 = D.source(mesh, p["Np"], p["rows"]).sum(0, keepdim=True).contiguous()
    rho, _ = op.solve(rho0, tol=1e-12)
    w = 1.0 / len(p["receiver"])
    g, dg = D.interior_density(mesh, p["Np"], p["receiver"], weights=w, mu=p["mu_t"])
    lam, dj, info = op.adjoint(rho, g, dg, tol=1e-12)
    # oracle gradient with its own operator derivative and its own solves
    ref = oracle_mod.assemble(m.verts, m.tets, p["mu"], 0.8, p["Np"], rtol=1e-12, with_derivative=True)
    b = oracle_mod.source_vector(m.verts, m.tets, p["rows"], p["Np"])
    rho_ref = oracle_mod.solve_dense(ref, b)
    gref, dgref = oracle_mod.receiver_functional(m.verts, m.tets, p["mu"], p["Np"], p["receiver"], nq=None)
    lam_ref, _ = oracle_mod.solve_gmres(ref, gref, tol=1e-14, trans=True)
    grad_ref = oracle_mod.gradient(ref, rho_ref, lam_ref, dgref, m.n_tets)
    got = dj[0].cpu().numpy()
    scale = np.abs(grad_ref).max()
    assert np.abs(got - grad_ref).max() <= 2e-5 * scale, (np.abs(got - grad_ref).max(), scale)
    # lambda: same adjoint equation on the GPU's operator, solved by LU
    blocks = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), m.n_tets)
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    same = oracle_mod.Operator(Np=p["Np"], blocks=blocks, dest=mesh.recv()[4 * t + fp].reshape(-1, 3).astype(np.int64))
    M = np.eye(same.nrows * same.nb) - oracle_mod.dense(same)
    lref = np.linalg.solve(M.T, g.cpu().numpy().ravel())
    assert np.linalg.norm(lam.cpu().numpy().ravel() - lref) <= 1e-9 * np.linalg.norm(lref)
    # adjoint identity lam^T rho0 = g^T rho on the GPU results
    assert float((lam * rho0[0]).sum()) == pytest.approx(float((g * rho[0]).sum()), rel=1e-9)


def test_adjoint_vs_central_differences(D, problem):
    import torch

    p = problem
    mesh = p["mesh"]
    Np = p["Np"]
    rho0 = D.source(mesh, Np, p["rows"]).sum(0, keepdim=True).contiguous()
    w = 1.0 / len(p["receiver"])

    def J(mu_vec):
        op = D.Operator(mesh, Np, mu=mu_vec, precision=D.F64)
        rho, _ = op.solve(rho0, method=D.GMRES, tol=1e-14)
        g, _ = D.interior_density(mesh, Np, p["receiver"], weights=w, mu=mu_vec)
        return float((g * rho[0]).sum())

    op = D.Operator(mesh, Np, mu=p["mu_t"], precision=D.F32)
    rho, _ = op.solve(rho0, tol=1e-12)
    g, dg = D.interior_density(mesh, Np, p["receiver"], weights=w, mu=p["mu_t"])
    _, dj, _ = op.adjoint(rho, g, dg, tol=1e-12)
    grad = dj[0].cpu().numpy()
    h = 1e-4
    for e in (0, 20, 31, 47):
        mp = p["mu_t"].clone()
        mp[e] += h
        mm = p["mu_t"].clone()
        mm[e] -= h
        fd = (J(mp) - J(mm)) / (2 * h)
        assert grad[e] == pytest.approx(fd, rel=1e-3, abs=1e-6 * np.abs(grad).max())


def test_autograd_function(D, problem):
    import torch

    p = problem
    mesh = p["mesh"]
    Np = p["Np"]
    rho0 = D.source(mesh, Np, p["rows"]).sum(0, keepdim=True).contiguous()
    mu = p["mu_t"].clone().requires_grad_(True)
    w = 1.0 / len(p["receiver"])
    g, _ = D.interior_density(mesh, Np, p["receiver"], weights=w, mu=p["mu_t"])
    rho = D.DFMSolve.apply(mesh, Np, mu, rho0, tol=1e-12)
    J = (rho[0] * g).sum()
    J.backward()
    op = D.Operator(mesh, Np, mu=p["mu_t"], precision=D.F32)
    r2, _ = op.solve(rho0, tol=1e-12)
    _, dj, _ = op.adjoint(r2, g, None, tol=1e-12)
    np.testing.assert_allclose(mu.grad.cpu().numpy(), dj[0].cpu().numpy(), rtol=1e-6,
                               atol=1e-9 * float(dj.abs().max()))
