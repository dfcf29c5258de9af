"""CUDA graphs of the preconditioner's Horner chains (dfm_hop_graphs).

The hops between the first and the last of a chain read and write only the
chain's scratch, so the solver captures them once per shape and replays the
graph.  Graphs change no arithmetic: solves and preconditioner applications
with graphs on and off agree bit for bit (single and batched right-hand
sides, forward and transposed, chunk-ordered and fragment-ordered copies),
the solver replays graphs when they are on and none when they are off, and
the graph-replayed solve matches LU of the same FP32 operator (the oracle's
dense solve of the GPU's own blocks)."""
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


def _dense_ref(oracle_mod, op, mesh, nt, Np):
    blocks = to_oracle_layout(op.blocks().double().cpu().numpy(), mesh.recv(), nt)
    t, f, fp = oracle_mod.pair_list(nt)
    dest = mesh.recv()[4 * t + fp].reshape(4 * nt, 3).astype(np.int64)
    ref = oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(blocks), dest=dest)
    return np.eye(ref.nrows * ref.nb) - oracle_mod.dense(ref)


@pytest.mark.parametrize("Np,R,trans,prec", [(4, 1, False, "e4m3"), (4, 8, False, "e4m3"), (8, 1, False, "e4m3"),
                                             (8, 8, False, "e4m3"), (4, 3, True, "e4m3"), (3, 5, True, "f16"),
                                             (4, 2, False, "bf16")])
def test_graph_replayed_solve_is_identical_and_matches_lu(D, oracle_mod, mesh161, Np, R, trans, prec):
    import torch

    verts, tets = mesh161
    nt = tets.shape[0]
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=0.2, precision=D.F32)
    rng = np.random.default_rng(Np * 10 + R)
    b = torch.tensor(rng.standard_normal((R, 4 * nt, op.nb)), dtype=torch.float64, device="cuda")
    pp = {"e4m3": D.FP8E4M3, "f16": D.F16, "bf16": D.BF16}[prec]
    kw = dict(tol=1e-10, transpose=trans, precond_precision=pp, poly_degree=12, restart=8)
    try:
        D.hop_graphs(0)
        r0 = D.hop_graph_replays()
        x_eager, info_eager = op.solve(b, **kw)
        assert D.hop_graph_replays() == r0
        D.hop_graphs(1)
        x_graph, info_graph = op.solve(b, **kw)
        replays = D.hop_graph_replays() - r0
    finally:
        D.hop_graphs(1)
    assert replays > 0
    assert torch.equal(x_eager, x_graph)
    assert (info_eager.iters, info_eager.outer) == (info_graph.iters, info_graph.outer)
    assert info_graph.resid <= 1e-10
    M = _dense_ref(oracle_mod, op, mesh, nt, Np)
    for r in range(R):
        want = np.linalg.solve(M.T if trans else M, b[r].cpu().numpy().ravel())
        assert np.linalg.norm(x_graph[r].cpu().numpy().ravel() - want) <= 1e-8 * np.linalg.norm(want)


@pytest.mark.parametrize("Np,R,prec", [(4, 1, "e4m3"), (4, 9, "e4m3"), (8, 16, "e4m3"), (5, 3, "f16"),
                                       (2, 2, "bf16")])
def test_graph_precond_is_identical(D, mesh161, Np, R, prec):
    """Repeated preconditioner applications (eager first, then captured and
    replayed wherever the scratch comes back at the same addresses) equal the
    eager chain bit for bit, after a reassembly too."""
    import torch

    verts, tets = mesh161
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=0.2, precision=D.F32)
    x = torch.randn((R, mesh.n_rows, op.nb), device="cuda", dtype=torch.float32)
    pp = {"e4m3": D.FP8E4M3, "f16": D.F16, "bf16": D.BF16}[prec]
    for mu in (0.2, 0.5):
        op.reassemble(mu)
        try:
            D.hop_graphs(0)
            want = op.precond(x, degree=7, precision=pp).clone()
        finally:
            D.hop_graphs(1)
        for _ in range(4):
            assert torch.equal(op.precond(x, degree=7, precision=pp), want)


def test_graph_launches_are_counted(D, mesh161):
    """A replayed graph counts its hops in the launch count: the same solve
    launches the same number of kernels with graphs on and off."""
    import torch

    verts, tets = mesh161
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, 4, mu=0.2, precision=D.F32)
    b = D.source(mesh, 4, [0, 5])
    op.solve(b, tol=1e-9, poly_degree=16, restart=8)  # first use of every shape (tuning, first chains)
    counts = []
    try:
        for mode in (0, 1):
            D.hop_graphs(mode)
            l0 = D.launch_count()
            op.solve(b, tol=1e-9, poly_degree=16, restart=8)
            torch.cuda.synchronize()
            counts.append(D.launch_count() - l0)
    finally:
        D.hop_graphs(1)
    assert counts[0] == counts[1]
