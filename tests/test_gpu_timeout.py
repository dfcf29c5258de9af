"""The time-out path of the pipelined kernels' bounded waits, exercised
without a fault: dfm_selftest_timeout runs a kernel whose wait is on a
barrier that nothing completes, with a limit of 1,000 polls (about a
millisecond), so it takes the same exit as a stalled copy and sets the
operator's error flag.  The host reads the flag with dfm_op_check_error (and
dfm_solve reads it after its iterations); the flag is cleared by reading and
the context stays usable."""
import numpy as np
import pytest

from gpu_helpers import need_gpu
from paper_1608_04607_gb300.inputs import kuhn_cube_mesh

pytestmark = pytest.mark.gpu


def test_timeout_flag_is_reported_and_cleared():
    need_gpu()
    import torch

    from paper_1608_04607_gb300 import dfm

    m = kuhn_cube_mesh(2, jitter=0.2, seed=3)
    mesh = dfm.Mesh(m.verts, m.tets, refl=0.9)
    op = dfm.Operator(mesh, 3, mu=0.1, precision=dfm.F32)
    op.check_error()  # nothing timed out yet
    dfm.selftest_timeout(op, polls=1000)
    with pytest.raises(dfm.DFMError) as e:
        op.check_error()
    assert e.value.code == dfm.DFM_ERR_TIMEOUT
    op.check_error()  # cleared by the read
    # a solve started after a time-out reports it
    rows = np.nonzero(mesh.recv() == np.arange(mesh.n_rows))[0][:1]
    rho0 = dfm.source(mesh, 3, rows)
    dfm.selftest_timeout(op, polls=1000)
    with pytest.raises(dfm.DFMError) as e:
        op.solve(rho0, tol=1e-8)
    assert e.value.code == dfm.DFM_ERR_TIMEOUT
    # the context is still usable and later work is correct
    rho, info = op.solve(rho0, tol=1e-10)
    x = torch.randn((mesh.n_rows, op.nb), device="cuda", dtype=torch.float64)
    y = op.apply(x)
    B = op.blocks().double()
    recv = torch.tensor(mesh.recv(), device="cuda", dtype=torch.int64)
    ref = torch.zeros_like(x)
    for R in range(mesh.n_rows):
        t, lp = int(recv[R]) // 4, int(recv[R]) % 4
        src = [4 * t + f for f in range(4) if f != lp]
        for k, J in enumerate(src):
            ref[R] += B[R, k] @ x[J]
    assert float((y - ref).abs().max()) <= 1e-10 * float(ref.abs().max())
    op.check_error()
