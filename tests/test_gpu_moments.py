"""Damping moments B^(k) = d^k B / d mu^k (uniform mu) and the combined
application / solve with per-right-hand-side damping (Taylor expansion about
mu_c), against the FP64 oracle:
 - B^(1) equals the oracle's derivative blocks dB/dmu;
 - sum_k (mu_r - mu_c)^k / k! B^(k) equals the oracle's B(mu_r) (truncation of
   order (|mu_r - mu_c| L)^K / K!, far below FP32 rounding here);
 - dfm_apply_combo equals the weighted sum of single applications;
 - dfm_solve_combo equals LU solves with the combined operators;
 - dfm_solve_damped (the library forms the Taylor weights from mu_r and the
   moments' mu_c) equals the oracle's solve with B(mu_r) assembled exactly.
"""
import math

import numpy as np
import pytest

from gpu_helpers import block_rel_err, need_gpu, to_oracle_layout
from paper_1608_04607_gb300.inputs import kuhn_cube_mesh

pytestmark = pytest.mark.gpu


def taylor_weights(mu_rhs, mu_c, K):
    """(mu_r - mu_c)^k / k!, restated here to check the combined operators."""
    mu_rhs = np.atleast_1d(np.asarray(mu_rhs, dtype=np.float64))
    return np.stack([(mu_rhs - mu_c) ** k / math.factorial(k) for k in range(K)], axis=1)


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    from paper_1608_04607_gb300 import dfm

    m = kuhn_cube_mesh(2, jitter=0.2, seed=12)
    mesh = dfm.Mesh(m.verts, m.tets, refl=0.95)
    Np, mu_c, K = 3, 0.105, 3
    ops = [dfm.Operator(mesh, Np, mu=mu_c, precision=dfm.F32, moment=k) for k in range(K)]
    return dfm, m, mesh, Np, mu_c, K, ops


def test_first_moment_is_oracle_derivative(setup, oracle_mod):
    dfm, m, mesh, Np, mu_c, K, ops = setup
    recv = mesh.recv()
    got = to_oracle_layout(ops[1].blocks().cpu().numpy(), recv, m.n_tets)
    ref = oracle_mod.assemble(m.verts, m.tets, np.full(m.n_tets, mu_c), 0.95, Np, rtol=1e-12, with_derivative=True)
    err = block_rel_err(got, ref.dblocks)
    assert err.max() <= 2e-5, err.max()


@pytest.mark.parametrize("mu_r", [0.01, 0.2])
def test_taylor_sum_matches_oracle(setup, oracle_mod, mu_r):
    dfm, m, mesh, Np, mu_c, K, ops = setup
    recv = mesh.recv()
    c = taylor_weights([mu_r], mu_c, K)[0]
    combo = sum(c[k] * to_oracle_layout(ops[k].blocks().cpu().numpy().astype(np.float64), recv, m.n_tets)
                for k in range(K))
    ref = oracle_mod.assemble(m.verts, m.tets, np.full(m.n_tets, mu_r), 0.95, Np, rtol=1e-12)
    err = block_rel_err(combo, ref.blocks)
    assert err.max() <= 1e-5, err.max()


def test_apply_combo_and_solve_combo(setup, oracle_mod):
    import torch

    dfm, m, mesh, Np, mu_c, K, ops = setup
    rng = np.random.default_rng(0)
    mu_rhs = rng.uniform(0.01, 0.2, 6)
    coef = taylor_weights(mu_rhs, mu_c, K)
    R = len(mu_rhs)
    x = torch.tensor(rng.standard_normal((R, mesh.n_rows, ops[0].nb)), device="cuda")
    y = dfm.apply_combo(ops, coef, x, x0=x, alpha=-1.0)
    for r in range(R):
        ref = x[r].clone()
        for k in range(K):
            ref -= coef[r, k] * ops[k].apply(x[r])
        assert float((y[r] - ref).abs().max()) <= 1e-12 * float(ref.abs().max())
    # solves: each right-hand side against LU with its own combined operator (FP32 blocks widened)
    recv = mesh.recv()
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    dest = recv[4 * t + fp].reshape(-1, 3).astype(np.int64)
    blocks = [to_oracle_layout(o.blocks().cpu().numpy(), recv, m.n_tets) for o in ops]
    rho0 = dfm.source(mesh, Np, np.nonzero(recv == np.arange(mesh.n_rows))[0][rng.integers(0, 48, R)])
    rho, info = dfm.solve_combo(ops, coef, rho0, tol=1e-10, batch=4)
    assert info.resid <= 1e-10
    for r in range(R):
        Br = oracle_mod.Operator(Np=Np, blocks=sum(coef[r, k] * blocks[k] for k in range(K)), dest=dest)
        ref = oracle_mod.solve_dense(Br, rho0[r].cpu().numpy())
        got = rho[r].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("precond", ["f16", "fp8"])
def test_solve_combo_with_low_precision_preconditioner(setup, oracle_mod, precond):
    """The flexible solve preconditions every right-hand side with p(B~_0),
    the polynomial on a low-precision copy of the first operator (B(mu_c));
    the solutions still match LU with each right-hand side's own operator."""
    dfm, m, mesh, Np, mu_c, K, ops = setup
    rng = np.random.default_rng(4)
    mu_rhs = rng.uniform(0.01, 0.2, 5)
    coef = taylor_weights(mu_rhs, mu_c, K)
    R = len(mu_rhs)
    recv = mesh.recv()
    t, f, fp = oracle_mod.pair_list(m.n_tets)
    dest = recv[4 * t + fp].reshape(-1, 3).astype(np.int64)
    blocks = [to_oracle_layout(o.blocks().cpu().numpy(), recv, m.n_tets) for o in ops]
    rho0 = dfm.source(mesh, Np, np.nonzero(recv == np.arange(mesh.n_rows))[0][rng.integers(0, 48, R)])
    pp = dfm.F16 if precond == "f16" else dfm.FP8E4M3
    rho, info = dfm.solve_combo(ops, coef, rho0, tol=1e-10, batch=4, precond_precision=pp)
    assert info.resid <= 1e-10
    for r in range(R):
        Br = oracle_mod.Operator(Np=Np, blocks=sum(coef[r, k] * blocks[k] for k in range(K)), dest=dest)
        ref = oracle_mod.solve_dense(Br, rho0[r].cpu().numpy())
        assert np.linalg.norm(rho[r].cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)


def test_solve_damped_matches_oracle_exact_damping(setup, oracle_mod):
    """Per-right-hand-side damping through the C ABI: dfm_solve_damped gets
    mu_r and the moments (assembled at mu_c), and its solutions match the
    oracle's LU solves with B(mu_r) assembled exactly (adaptive quadrature to
    1e-12, no Taylor expansion).  Four moments keep the truncation
    ((|mu_r - mu_c| L)^4 / 4! < 1e-6 per entry here) below the FP32 entry
    error; the remaining difference is the FP32 assembly's (<= 1e-5 per block)
    times the conditioning of I - B, within 1e-4."""
    dfm, m, mesh, Np, mu_c, _, _ = setup
    ops = [dfm.Operator(mesh, Np, mu=mu_c, precision=dfm.F32, moment=k) for k in range(4)]
    recv = mesh.recv()
    rng = np.random.default_rng(8)
    mu_rhs = np.array([0.01, 0.2, 0.105, 0.06])
    R = len(mu_rhs)
    rows = np.nonzero(recv == np.arange(mesh.n_rows))[0][rng.integers(0, 48, R)]
    rho0 = dfm.source(mesh, Np, rows)
    rho, info = dfm.solve_damped(ops, mu_rhs, rho0, tol=1e-10, batch=2)
    assert info.resid <= 1e-10
    for r in range(R):
        ref_op = oracle_mod.assemble(m.verts, m.tets, np.full(m.n_tets, mu_rhs[r]), 0.95, Np, rtol=1e-12)
        ref = oracle_mod.solve_dense(ref_op, oracle_mod.source_vector(m.verts, m.tets, rows[r:r + 1], Np))
        got = rho[r].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref), np.linalg.norm(got - ref) / np.linalg.norm(ref)
    # moments given in the wrong order, or a moment at another damping, are refused
    with pytest.raises(dfm.DFMError):
        dfm.solve_damped([ops[1], ops[0]], mu_rhs, rho0)
    other = dfm.Operator(mesh, Np, mu=0.2, precision=dfm.F32, moment=1)
    with pytest.raises(dfm.DFMError):
        dfm.solve_damped([ops[0], other], mu_rhs, rho0)
    with pytest.raises(dfm.DFMError):
        dfm.solve_damped(ops[:2], np.array([0.1, -0.1, 0.1, 0.1]), rho0)
