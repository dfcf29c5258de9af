"""Host-side argument checks of the Python binding: coefficient tensors are
checked for dtype and shape before their pointers cross the C ABI (the
library sees only pointers and counts, so a short buffer would be read out of
bounds).  CPU only: every case here is rejected before any library call."""
import types

import pytest

torch = pytest.importorskip("torch")

from paper_1608_04607_gb300 import dfm  # noqa: E402

ROWS, NB = 24, 6


def _fake_op():
    return types.SimpleNamespace(n_rows=ROWS, nb=NB, _torch=torch, _h=None, _p=None,
                                 mesh=types.SimpleNamespace(n_tets=ROWS // 4))


def _bad(fn, *a, **k):
    with pytest.raises(dfm.DFMError) as e:
        fn(*a, **k)
    assert e.value.code == dfm.DFM_ERR_ARG


def test_vec_accepts_both_layouts():
    assert dfm._vec(torch.zeros(ROWS, NB, dtype=torch.float64), ROWS, NB, (torch.float64,), "x") == 1
    assert dfm._vec(torch.zeros(3, ROWS, NB, dtype=torch.float32), ROWS, NB,
                    (torch.float32, torch.float64), "x") == 3


@pytest.mark.parametrize("t", [
    torch.zeros(ROWS, NB, dtype=torch.float32),           # wrong dtype
    torch.zeros(ROWS, NB + 1, dtype=torch.float64),       # wrong basis size
    torch.zeros(ROWS - 4, NB, dtype=torch.float64),       # wrong row count
    torch.zeros(ROWS * NB, dtype=torch.float64),          # flattened
    torch.zeros(1, 2, ROWS, NB, dtype=torch.float64),     # extra dimension
])
def test_vec_rejects(t):
    _bad(dfm._vec, t, ROWS, NB, (torch.float64,), "x")


def test_like():
    ref = torch.zeros(2, ROWS, NB, dtype=torch.float64)
    dfm._like(None, ref, "x0")
    dfm._like(torch.zeros_like(ref), ref, "x0")
    _bad(dfm._like, torch.zeros(1, ROWS, NB, dtype=torch.float64), ref, "x0")
    _bad(dfm._like, torch.zeros(2, ROWS, NB, dtype=torch.float32), ref, "x0")


def test_operator_methods_check_before_the_abi():
    op = _fake_op()
    f64 = torch.zeros(ROWS, NB, dtype=torch.float64)
    _bad(dfm.Operator.solve, op, torch.zeros(ROWS, NB, dtype=torch.float32))
    _bad(dfm.Operator.solve, op, f64, x0=torch.zeros(2, ROWS, NB, dtype=torch.float64))
    _bad(dfm.Operator.apply, op, torch.zeros(ROWS, NB + 1))
    _bad(dfm.Operator.apply, op, f64, x0=torch.zeros(ROWS, NB, dtype=torch.float32))
    _bad(dfm.Operator.apply, op, f64, out=torch.zeros(2, ROWS, NB, dtype=torch.float64))
    _bad(dfm.Operator.precond, op, torch.zeros(ROWS + 4, NB))
    _bad(dfm.Operator.adjoint, op, f64, torch.zeros(1, ROWS, NB, dtype=torch.float64))
    _bad(dfm.Operator.adjoint, op, f64, f64, dgvec=torch.zeros(ROWS, NB))
    ops = [op, op]
    _bad(dfm.apply_combo, ops, [[1.0, 0.5]], torch.zeros(ROWS, NB - 1))
    _bad(dfm.apply_combo, ops, [[1.0, 0.5, 0.2]], f64)
    _bad(dfm.solve_combo, ops, [[1.0, 0.5]], torch.zeros(ROWS, NB))
    mesh = types.SimpleNamespace(n_rows=ROWS, n_tets=ROWS // 4, handle=None)
    _bad(dfm.tet_density, mesh, 2, torch.zeros(1, ROWS, NB, dtype=torch.float64), f64)
    _bad(dfm.tet_density, mesh, 2, f64, torch.zeros(ROWS, NB))
    _bad(dfm.interior_density, mesh, 2, [0], gvec=torch.zeros(ROWS, NB - 1, dtype=torch.float64),
         dgvec=torch.zeros(ROWS, NB, dtype=torch.float64))


def test_damping_field_length_is_checked():
    """A per-tet damping tensor must hold one value per tet: the library reads
    n_tets values through the pointer.  A 0-dim tensor means uniform damping."""
    op = _fake_op()
    for bad in (torch.zeros(ROWS // 4 - 1, dtype=torch.float64), torch.zeros(ROWS, dtype=torch.float64),
                torch.zeros(2, ROWS // 4, dtype=torch.float64)):
        _bad(dfm.Operator._params, op, 2, bad, dfm.F32, 0, 0.0)
    p = dfm.Operator._params(op, 2, torch.tensor(0.25, dtype=torch.float64), dfm.F32, 0, 0.0)
    assert p.mu is None and p.mu_uniform == 0.25


def test_solve_damped_checks_before_the_abi():
    op = _fake_op()
    rho0 = torch.zeros(3, ROWS, NB, dtype=torch.float64)
    _bad(dfm.solve_damped, [op], [0.1, 0.2], rho0)          # one damping per right-hand side
    _bad(dfm.solve_damped, [op], [0.1, 0.2, 0.3], rho0.float())
