"""Parity at the full 48,000-tet workload, in the launch configuration the
benchmark times (FP32 operator, GMRES-IR to 1e-8):
 - 200 sampled blocks against the oracle computed one by one (1e-5 of the
   block max-norm);
 - the solution's FP64 residual recomputed by the oracle's own operator
   application on the assembled blocks (a property that holds at any size);
 - the mass balance w^T (I - B) rho = w^T rho0 with w = sqrt|T| on (0,0).
"""
import numpy as np
import pytest

from gpu_helpers import block_rel_err, need_gpu, to_oracle_layout
from paper_1608_04607_gb300.inputs import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    from paper_1608_04607_gb300 import dfm

    w = workload("kuhn20_np4")
    m = w["mesh"]
    mesh = dfm.Mesh(m.verts, m.tets, refl=w["refl"])
    op = dfm.Operator(mesh, w["Np"], mu=float(w["mu"][0]), precision=dfm.F32)
    return dfm, w, m, mesh, op


def test_sampled_blocks(setup, oracle_mod):
    dfm, w, m, mesh, op = setup
    recv = mesh.recv()
    vals = op.blocks().cpu().numpy()
    rng = np.random.default_rng(42)
    topo = oracle_mod.topology(m.tets)
    np.testing.assert_array_equal(recv, topo.recv)
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    sel = rng.choice(t.size, 200, replace=False)
    ref, _, q, _ = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, w["mu"], w["refl"], w["Np"], t[sel], f[sel],
                                               fp[sel], rtol=1e-12)
    R = recv[4 * t[sel] + fp[sel]]
    slot = f[sel] - (f[sel] > fp[sel])
    got = vals[R, slot]
    err = block_rel_err(got, ref)
    assert err.max() <= 1e-5, err.max()


def test_solution_residual_and_balance(setup, oracle_mod):
    dfm, w, m, mesh, op = setup
    rho0 = dfm.source(mesh, w["Np"], w["sources"])
    rho, info = op.solve(rho0, method=dfm.GMRES_IR, tol=1e-8)
    assert info.resid <= 1e-8
    blocks = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), m.n_tets)
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    dest = mesh.recv()[4 * t + fp].reshape(-1, 3).astype(np.int64)
    same = oracle_mod.Operator(Np=w["Np"], blocks=np.ascontiguousarray(blocks), dest=dest)
    x = rho[0].cpu().numpy()
    b = rho0[0].cpu().numpy()
    assert oracle_mod.residual(same, x, b) <= 1.2e-8
    A = oracle_mod.face_areas(m.verts, m.tets)
    wv = np.zeros_like(b)
    wv[:, 0] = np.sqrt(A)
    lhs = np.sum(wv * (x - oracle_mod.apply(same, x)))
    assert lhs == pytest.approx(np.sum(wv * b), rel=1e-6)
