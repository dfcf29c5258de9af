"""The C ABI library builds, loads and exports every entry point declared in
include/dfm.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dfm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"^\s*#.*$", "", src, flags=re.M)
    return sorted(set(re.findall(r"^[ \t]*(?!typedef)[A-Za-z_][\w \t\*]*?\b(dfm_\w+)[ \t]*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dfm_mesh_create", "dfm_assemble", "dfm_solve", "dfm_apply", "dfm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1608_04607_gb300 import build, dfm

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers the whole header
    assert set(declared_functions()) == set(dfm.SIGNATURES)
    assert lib.dfm_version


def test_null_handles_are_rejected_on_the_host():
    """Argument checks run before any CUDA call: NULL handles and empty counts
    come back as DFM_ERR_ARG with a message, here without a GPU."""
    from paper_1608_04607_gb300 import dfm

    L = dfm.load()
    ARG = dfm.DFM_ERR_ARG
    one = (ctypes.c_int64 * 1)(0)
    calls = {
        "dfm_source": lambda: L.dfm_source(None, 2, one, 1, None, None),
        "dfm_source_directed": lambda: L.dfm_source_directed(None, 2, one, None, 1, 0, None, None),
        "dfm_point_source": lambda: L.dfm_point_source(None, 2, one, 1, None, 0.0, 1.0, 0, None, None),
        "dfm_tet_density": lambda: L.dfm_tet_density(None, 2, None, None, 1, None, None),
        "dfm_interior_density": lambda: L.dfm_interior_density(None, 2, None, 0.0, one, None, 1, 0, None, None,
                                                               None),
        "dfm_apply": lambda: L.dfm_apply(None, None, None, None, 1, 1.0, 0, dfm.F32, None),
        "dfm_precond_apply": lambda: L.dfm_precond_apply(None, dfm.F16, 4, 0, None, None, 1, None),
        "dfm_solve": lambda: L.dfm_solve(None, None, 1, None, None, None, None),
        "dfm_solve_combo": lambda: L.dfm_solve_combo(None, 0, None, None, 1, None, None, None, None),
        "dfm_solve_damped": lambda: L.dfm_solve_damped(None, 0, None, None, 1, None, None, None, None),
        "dfm_op_check_error": lambda: L.dfm_op_check_error(None, None),
        "dfm_selftest_timeout": lambda: L.dfm_selftest_timeout(None, 10, None),
        "dfm_adjoint": lambda: L.dfm_adjoint(None, None, None, 1, None, None, None, None, None, None, None),
        "dfm_op_info": lambda: L.dfm_op_info(None, None),
        "dfm_mesh_info": lambda: L.dfm_mesh_info(None, None),
    }
    for name, call in calls.items():
        assert call() == ARG, name
        assert L.dfm_last_error().decode().startswith(name), (name, L.dfm_last_error())


def test_assembly_parameters_are_checked_before_the_mesh_is_touched():
    """Np out of range (0..20; above 8 FP32 blocks only), an unknown precision, negative or NaN damping, and out-of-range
    quadrature settings are refused by dfm_assemble before it reads the mesh or calls
    CUDA (the mesh handle here is a zeroed host buffer that is never read)."""
    from paper_1608_04607_gb300 import dfm

    L = dfm.load()
    fake_mesh = ctypes.create_string_buffer(4096)
    out = ctypes.c_void_p()
    good = dict(Np=4, mu=None, mu_uniform=0.1, quad_order=0, max_patch_deg=0.0, precision=dfm.F32, moment=0)
    cases = [dict(Np=21), dict(Np=-1), dict(Np=9, precision=dfm.BF16), dict(Np=20, precision=dfm.F64),
             dict(Np=dfm.basis(9, 1)), dict(Np=dfm.basis(4, 2)), dict(Np=dfm.basis(4, 1), precision=dfm.BF16),
             dict(Np=dfm.basis(4, 1), moment=1),
             dict(precision=7), dict(mu_uniform=-0.1), dict(mu_uniform=float("nan")),
             dict(quad_order=33), dict(max_patch_deg=5.0), dict(moment=4)]
    for bad in cases:
        p = dfm.Params(**{**good, **bad})
        rc = L.dfm_assemble(ctypes.cast(fake_mesh, ctypes.c_void_p), ctypes.byref(p), None, ctypes.byref(out))
        assert rc in (dfm.DFM_ERR_ARG, dfm.DFM_ERR_UNSUPPORTED), bad
        assert L.dfm_last_error().decode().startswith("dfm_assemble"), bad
        assert not out.value


def test_hop_graph_switch_on_the_host():
    """dfm_hop_graphs only flips a process-wide switch: no CUDA call."""
    from paper_1608_04607_gb300 import dfm

    L = dfm.load()
    assert L.dfm_hop_graphs(-1) == 1
    assert L.dfm_hop_graphs(2) == dfm.DFM_ERR_ARG
    try:
        assert L.dfm_hop_graphs(0) == 0 and L.dfm_hop_graphs(-1) == 0
    finally:
        assert L.dfm_hop_graphs(1) == 1
    assert L.dfm_hop_graph_replays() == 0
