"""GPU parity of the low-precision polynomial preconditioner
(dfm_precond_apply, the hops of the flexible inner solve) with the oracle.

The preconditioner is z = sum_{k<d} B~^k x, B~ the FP16 or BF16 rounding (to
nearest, ties to even) of the FP32 blocks, or s_R times their e4m3 rounding
relative to a per-row scale s_R = max |row entry| / 448.  The oracle
evaluates the same sum in FP64 from the GPU's FP32 blocks rounded the same way
on the host, so the only difference left is the kernels' arithmetic (see
TOL).  The mesh drops one tet of the Kuhn cube (161 tets), so the last tile
of rows is ragged for every basis size; N_p = 2, 4, 5 give 6, 15, 21
functions, N_p = 3 and 8 give 10 and 45 (padded widths 8, 16, 24, 16, 48).
With a padded width that is a multiple of 16 (N_p = 3, 4, 8 with the FP16
and e4m3 copies) the hops run on tensor cores on the fragment-ordered copy:
R <= 3 one right-hand side per launch, R >= 4 in groups of 8 (R = 4 and 5
fill part of one group, 9 one group and part of a second, 16 two full groups
in one launch, 17 a second launch for the third group)."""
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


# The BF16 copy runs on FP32 vectors with FP32 accumulation: only FP32
# rounding separates it from the oracle (<= 2e-5 of max |z| over 4 hops).  The
# FP16 and e4m3 copies run on FP16 vectors (x scaled by a power of two) and
# sum each block's products in packed FP16 before adding the three blocks in
# FP32: per hop the vector is rounded to FP16 (relative 2^-11) and each lane
# adds 2 NBP/8 <= 6 products with one rounding each, so 5 hops stay within
# 3e-3 of max |z|, while a wrong block, slot or scale gives errors of order 1.
TOL = {"bf16": 2e-5, "f16": 3e-3, "e4m3": 3e-3}


def _round_f16(a32):
    return np.asarray(a32, dtype=np.float32).astype(np.float16).astype(np.float64)


def _round_bf16(a32):
    u = np.ascontiguousarray(a32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _e4m3(v):
    """Round float32 values to e4m3 (to nearest, ties to even; saturate at
    448): 3 fraction bits, normal exponents down to 2^-6, subnormal spacing
    2^-9."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    _, ex = np.frexp(a)  # a = f 2^ex, f in [0.5, 1)
    e = np.maximum(ex - 1, -6)
    spacing = np.ldexp(1.0, e - 3)
    q = np.round(a / spacing) * spacing
    return np.sign(v) * np.minimum(q, 448.0)


def _round_e4m3_rows(b32, recv, nt):
    """The e4m3 copy in the operator's row layout b32[row, slot, a, b]:
    s_R = max |entry of row R| / 448 (FP32), q = e4m3(v / s_R) with v / s_R
    rounded to FP32, value = s_R q."""
    b32 = np.asarray(b32, dtype=np.float32)
    mx = np.abs(b32).reshape(b32.shape[0], -1).max(axis=1).astype(np.float32)
    s = np.where(mx > 0, mx / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    ratio = (b32 / s[:, None, None, None]).astype(np.float32)
    return _e4m3(ratio) * s.astype(np.float64)[:, None, None, None]


@pytest.fixture(scope="module")
def mesh161():
    m = kuhn_cube_mesh(3, jitter=0.2, seed=8)
    return m.verts, np.ascontiguousarray(m.tets[:-1])


@pytest.mark.parametrize("Np,R", [(2, 3), (3, 3), (3, 4), (4, 1), (4, 3), (4, 9), (4, 17), (5, 3), (8, 5), (8, 16)])
@pytest.mark.parametrize("prec", ["f16", "bf16", "e4m3"])
def test_precond_matches_oracle_on_rounded_blocks(D, oracle_mod, mesh161, Np, R, prec):
    import torch

    verts, tets = mesh161
    nt = tets.shape[0]
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=0.2, precision=D.F32)
    b32 = op.blocks().cpu().numpy()
    if prec == "e4m3":
        rounded = _round_e4m3_rows(b32, mesh.recv(), nt)
    else:
        rounded = _round_f16(b32) if prec == "f16" else _round_bf16(b32)
    blocks = to_oracle_layout(rounded, mesh.recv(), nt)
    t, f, fp = oracle_mod.pair_list(nt)
    dest = mesh.recv()[4 * t + fp].reshape(4 * nt, 3).astype(np.int64)
    ref_op = oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(blocks), dest=dest)
    rng = np.random.default_rng(Np)
    x = rng.standard_normal((R, 4 * nt, op.nb)).astype(np.float32)
    xt = torch.tensor(x, device="cuda")
    for d in (1, 2, 5):
        z = op.precond(xt, degree=d, precision={"f16": D.F16, "bf16": D.BF16, "e4m3": D.FP8E4M3}[prec])
        z = z.cpu().numpy()
        for r in range(R):
            xr = x[r].astype(np.float64)
            zr = xr.copy()
            for _ in range(d - 1):
                zr = xr + oracle_mod.apply(ref_op, zr)
            assert np.abs(z[r] - zr).max() <= TOL[prec] * np.abs(zr).max(), (d, r)


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


@pytest.mark.parametrize("prec", ["f16", "e4m3"])
def test_precond_fp16_vectors_follow_the_input_scale(D, mesh161, prec):
    """The FP16 hop vectors hold x times a power of two chosen from max |x|,
    so the result scales with x across the FP16 range and beyond it."""
    import torch

    verts, tets = mesh161
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, 4, mu=0.2, precision=D.F32)
    p = D.F16 if prec == "f16" else D.FP8E4M3
    x = torch.randn((4 * tets.shape[0], op.nb), device="cuda", dtype=torch.float32)
    z = op.precond(x, degree=6, precision=p)
    for s in (2.0 ** 40, 2.0 ** -40):
        zs = op.precond(x * s, degree=6, precision=p)
        assert torch.isfinite(zs).all()
        assert float((zs / s - z).abs().max()) <= 1e-6 * float(z.abs().max())


def _round_e4m3_columns(blocks32):
    """The transposed e4m3 copy: row J of B^T holds the three blocks column J
    sends (the oracle's column layout blocks[J]), so its scale is the largest
    entry of blocks[J]; values rounded as in _round_e4m3_rows."""
    b32 = np.asarray(blocks32, dtype=np.float32)
    mx = np.abs(b32).reshape(b32.shape[0], -1).max(axis=1).astype(np.float32)
    s = np.where(mx > 0, mx / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    ratio = (b32 / s[:, None, None, None]).astype(np.float32)
    return _e4m3(ratio) * s.astype(np.float64)[:, None, None, None]


@pytest.mark.parametrize("Np,R", [(2, 1), (4, 1), (4, 3), (4, 9), (8, 1), (8, 5)])
@pytest.mark.parametrize("prec", ["f16", "bf16", "e4m3"])
def test_transposed_precond_matches_oracle(D, oracle_mod, mesh161, Np, R, prec):
    """z = sum_{k<d} (B~^T)^k x on the transposed copy (the adjoint solve's
    preconditioner) against the oracle's transposed application of the same
    rounded blocks."""
    import torch

    verts, tets = mesh161
    nt = tets.shape[0]
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=0.2, precision=D.F32)
    cols32 = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), nt).astype(np.float32)
    if prec == "e4m3":
        rounded = _round_e4m3_columns(cols32)
    else:
        rounded = _round_f16(cols32) if prec == "f16" else _round_bf16(cols32)
    t, f, fp = oracle_mod.pair_list(nt)
    dest = mesh.recv()[4 * t + fp].reshape(4 * nt, 3).astype(np.int64)
    ref_op = oracle_mod.Operator(Np=Np, blocks=np.ascontiguousarray(rounded), dest=dest)
    rng = np.random.default_rng(10 + Np)
    x = rng.standard_normal((R, 4 * nt, op.nb)).astype(np.float32)
    xt = torch.tensor(x, device="cuda")
    for d in (2, 5):
        z = op.precond(xt, degree=d, precision={"f16": D.F16, "bf16": D.BF16, "e4m3": D.FP8E4M3}[prec],
                       transpose=True).cpu().numpy()
        for r in range(R):
            xr = x[r].astype(np.float64)
            zr = xr.copy()
            for _ in range(d - 1):
                zr = xr + oracle_mod.apply(ref_op, zr, trans=True)
            assert np.abs(z[r] - zr).max() <= TOL[prec] * np.abs(zr).max(), (d, r)


@pytest.mark.parametrize("prec", ["f16", "e4m3"])
def test_transposed_solve_with_low_precision_preconditioner(D, oracle_mod, mesh161, prec):
    """(I - B)^T x = b with the flexible solve preconditioned on the transposed
    copy matches LU of the same FP32 operator."""
    import torch

    verts, tets = mesh161
    nt = tets.shape[0]
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, 4, mu=0.2, precision=D.F32)
    blocks = to_oracle_layout(op.blocks().cpu().numpy(), mesh.recv(), nt)
    t, f, fp = oracle_mod.pair_list(nt)
    dest = mesh.recv()[4 * t + fp].reshape(4 * nt, 3).astype(np.int64)
    ref_op = oracle_mod.Operator(Np=4, blocks=np.ascontiguousarray(blocks), dest=dest)
    M = np.eye(ref_op.nrows * ref_op.nb) - oracle_mod.dense(ref_op)
    rng = np.random.default_rng(3)
    b = torch.tensor(rng.standard_normal((2, 4 * nt, op.nb)), dtype=torch.float64, device="cuda")
    x, info = op.solve(b, tol=1e-10, transpose=True, precond_precision=D.F16 if prec == "f16" else D.FP8E4M3)
    assert info.resid <= 1e-10
    for r in range(2):
        want = np.linalg.solve(M.T, b[r].cpu().numpy().ravel())
        assert np.linalg.norm(x[r].cpu().numpy().ravel() - want) <= 1e-8 * np.linalg.norm(want)


@pytest.mark.parametrize("Np,R", [(8, 1), (4, 9)])
def test_autotuned_hops_are_identical_and_reported(D, mesh161, Np, R):
    """The autotuner times the candidate tile geometries of the tensor-core
    hop on the first launch of a shape and keeps the fastest; geometry changes
    no arithmetic, so hops with tuning on and off agree bit for bit, and the
    report names the shape, its candidates and the fastest as the choice."""
    import torch

    verts, tets = mesh161
    mesh = D.Mesh(verts, tets, refl=0.9)
    op = D.Operator(mesh, Np, mu=0.2, precision=D.F32)
    x = torch.randn((R, mesh.n_rows, op.nb), device="cuda", dtype=torch.float32)
    try:
        D.autotune(0)
        z0 = op.precond(x, degree=4, precision=D.FP8E4M3)
        D.autotune(2)
        z1 = op.precond(x, degree=4, precision=D.FP8E4M3)
        z2 = op.precond(x, degree=4, precision=D.FP8E4M3)
    finally:
        D.autotune(1)
    assert torch.equal(z0, z1) and torch.equal(z1, z2)
    rep = [e for e in D.autotune_report() if e["rows"] == mesh.n_rows and e["nb"] == op.nb]
    assert rep, D.autotune_report()
    for e in rep:
        assert e["kernel"] == "hop_frag" and len(e["tried"]) >= 2
        best = min(e["tried"], key=lambda t: t[2])
        assert [e["chosen"]["rows_per_tile"], e["chosen"]["stages"]] == best[:2]
