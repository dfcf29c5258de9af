"""GPU parity of mesh set-up, quadrature tables and operator assembly against
the FP64 oracle (all calls go through the C ABI of libdfm).

Tolerances: the GPU integrates each direction patch with a fixed Gauss rule
(order Np + 6 after splitting patches to <= 60 degrees), which the oracle's
order doubling shows to be accurate to ~3e-7 of the block max-norm; FP32
arithmetic adds ~1e-6.  Operator entries must match to 1e-5 relative to the
block max-norm in FP32 (the method's stated entry tolerance) and 2e-6 in FP64.
"""
import numpy as np
import pytest

from gpu_helpers import block_rel_err, need_gpu, to_oracle_layout
from paper_1608_04607_gb300.inputs import kuhn_cube_mesh, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    need_gpu()
    from paper_1608_04607_gb300 import dfm

    dfm.load()
    return dfm


def test_gauss_legendre_on_device(D):
    for q in (1, 2, 5, 10, 16, 32, 64):
        x, w = D.gauss_legendre(q)
        xr, wr = np.polynomial.legendre.leggauss(q)
        np.testing.assert_allclose(x.cpu().numpy(), xr, atol=2e-15)
        np.testing.assert_allclose(w.cpu().numpy(), wr, atol=2e-15)


def test_mesh_topology_matches_oracle(D, oracle_mod):
    for n, jit in ((1, 0.0), (3, 0.2), (6, 0.2)):
        m = kuhn_cube_mesh(n, jitter=jit, seed=4)
        mesh = D.Mesh(m.verts, m.tets, refl=0.9)
        topo = oracle_mod.topology(m.tets)
        np.testing.assert_array_equal(mesh.recv(), topo.recv)
        info = mesh.info()
        assert info.n_boundary_rows == 12 * n * n
        assert info.total_volume == pytest.approx(1.0, rel=1e-12)


def test_mesh_errors_are_reported(D):
    m = kuhn_cube_mesh(1, jitter=0.0)
    bad = m.tets.copy()
    bad[0, 0] = 99
    with pytest.raises(D.DFMError) as e:
        D.Mesh(m.verts, bad)
    assert e.value.code == D.DFM_ERR_MESH
    # three tets sharing one face
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 1]], float)
    T = np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]], np.int32)
    with pytest.raises(D.DFMError) as e:
        D.Mesh(V, T)
    assert e.value.code == D.DFM_ERR_MESH
    # flat tet
    V2 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], float)
    with pytest.raises(D.DFMError) as e:
        D.Mesh(V2, np.array([[0, 1, 2, 3]], np.int32))
    assert e.value.code == D.DFM_ERR_MESH
    with pytest.raises(D.DFMError) as e:
        D.Mesh(m.verts, m.tets, refl=1.5)
    assert e.value.code == D.DFM_ERR_ARG


def _oracle_op(oracle_mod, m, mu, refl, Np, rtol=1e-12):
    return oracle_mod.assemble(m.verts, m.tets, mu, refl, Np, rtol=rtol)


@pytest.mark.parametrize("prec,tol", [(0, 2e-6), (1, 1e-5)])
def test_assembly_single_cube(D, oracle_mod, prec, tol):
    w = workload("kuhn1_np2")
    m = w["mesh"]
    mesh = D.Mesh(m.verts, m.tets, refl=w["refl"])
    op = D.Operator(mesh, w["Np"], mu=0.1, precision=prec)
    got = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), m.n_tets)
    ref = _oracle_op(oracle_mod, m, w["mu"], w["refl"], w["Np"])
    err = block_rel_err(got, ref.blocks)
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("Np", [0, 1, 3, 4, 6, 8])
def test_assembly_jittered_fp32(D, oracle_mod, Np):
    import torch

    m = kuhn_cube_mesh(2, jitter=0.2, seed=21)
    rng = np.random.default_rng(Np)
    mu = rng.uniform(0.0, 0.4, m.n_tets)
    mesh = D.Mesh(m.verts, m.tets, refl=0.8)
    op = D.Operator(mesh, Np, mu=torch.tensor(mu, device="cuda"), precision=D.F32)
    got = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), m.n_tets)
    topo = oracle_mod.topology(m.tets)
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    sel = np.arange(12 * m.n_tets) if Np <= 4 else rng.choice(12 * m.n_tets, 96, replace=False)
    ref, _, q, _ = oracle_mod.blocks_for_pairs(m.verts, m.tets, topo, mu, 0.8, Np, t[sel], f[sel], fp[sel],
                                               rtol=1e-12)
    err = block_rel_err(got.reshape(-1, got.shape[2], got.shape[3])[sel], ref)
    assert err.max() <= 1e-5, (err.max(), np.argmax(err))


def test_assembly_is_deterministic_and_reassembles(D):
    import torch

    m = kuhn_cube_mesh(3, jitter=0.2, seed=2)
    mesh = D.Mesh(m.verts, m.tets, refl=0.95)
    op = D.Operator(mesh, 4, mu=0.05)
    a = op.blocks().clone()
    op.reassemble(0.3)
    b = op.blocks().clone()
    op.reassemble(0.05)
    c = op.blocks()
    assert torch.equal(a, c)
    assert not torch.equal(a, b)
