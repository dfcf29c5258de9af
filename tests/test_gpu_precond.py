"""GPU parity of the 16-bit polynomial preconditioner (dfm_precond_apply,
the hops of the flexible inner solve) with the oracle.

The preconditioner is z = sum_{k<d} B~^k x, B~ the FP16 or BF16 rounding (to
nearest, ties to even) of the FP32 blocks.  The oracle evaluates the same sum
in FP64 from the GPU's FP32 blocks rounded the same way on the host, so the
only difference left is FP32 arithmetic in the kernels: relative error
<= 2e-5 of max |z| for up to 5 hops.  The mesh drops one tet of the Kuhn cube
(161 tets), so the last tile of rows is ragged for every basis size; N_p = 2,
4, 5 give 6, 15, 21 functions (padded widths 8, 16, 24: 16, 8 and 5 rows per
tile)."""
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


def _round_f16(a32):
    return np.asarray(a32, dtype=np.float32).astype(np.float16).astype(np.float64)


def _round_bf16(a32):
    u = np.ascontiguousarray(a32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def mesh161():
    m = kuhn_cube_mesh(3, jitter=0.2, seed=8)
    return m.verts, np.ascontiguousarray(m.tets[:-1])


@pytest.mark.parametrize("Np", [2, 4, 5])
@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_precond_matches_oracle_on_rounded_blocks(D, oracle_mod, mesh161, Np, prec):
    import torch

    verts, tets = mesh161
    nt = tets.shape[0]
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=0.2, precision=D.F32)
    b32 = op.blocks().cpu().numpy()
    rounded = _round_f16(b32) if prec == "f16" else _round_bf16(b32)
    blocks = to_oracle_layout(rounded, mesh.recv(), nt)
    t, f, fp = oracle_mod.pair_list(nt)
    dest = mesh.recv()[4 * t + fp].reshape(4 * nt, 3).astype(np.int64)
    ref_op = oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(blocks), dest=dest)
    rng = np.random.default_rng(Np)
    R = 3
    x = rng.standard_normal((R, 4 * nt, op.nb)).astype(np.float32)
    xt = torch.tensor(x, device="cuda")
    for d in (1, 2, 5):
        z = op.precond(xt, degree=d, precision=D.F16 if prec == "f16" else D.BF16).cpu().numpy()
        for r in range(R):
            xr = x[r].astype(np.float64)
            zr = xr.copy()
            for _ in range(d - 1):
                zr = xr + oracle_mod.apply(ref_op, zr)
            assert np.abs(z[r] - zr).max() <= 2e-5 * np.abs(zr).max(), (d, r)


def test_precond_tracks_reassembly_and_rejects_bad_arguments(D, mesh161):
    """The 16-bit copy is rebuilt after an assembly; degree and aliasing are
    checked before any launch."""
    import torch

    verts, tets = mesh161
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, 4, mu=0.2, precision=D.F32)
    x = torch.randn((4 * tets.shape[0], op.nb), device="cuda", dtype=torch.float32)
    z1 = op.precond(x, degree=3).clone()
    op.reassemble(0.6)
    z2 = op.precond(x, degree=3)
    ref = op.apply(op.apply(x, x0=x), x0=x)  # x + B (x + B x) with the FP32 blocks
    assert not torch.equal(z1, z2)
    assert float((z2 - ref).abs().max()) <= 1e-2 * float(ref.abs().max())
    with pytest.raises(RuntimeError):
        op.precond(x, degree=0)
    with pytest.raises(RuntimeError):
        op.precond(x, degree=65)
    with pytest.raises(RuntimeError):
        op.precond(x, degree=2, out=x)
