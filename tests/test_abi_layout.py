"""The Python binding's ctypes mirrors of the structs of include/dfm.h have
the C layout: every field at the C offset and the same size (a C program
compiled against the header prints them).  No GPU needed."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_ctypes_structs_match_the_header():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1608_04607_gb300 import dfm

    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "abi_layout_check")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_layout_check.c"),
                    "-o", exe], check=True)
    lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    c_layout = {}
    for ln in lines:
        if ln.strip():
            s, f, v = ln.split()
            c_layout.setdefault(s, {})[f] = int(v)
    mirrors = {"dfm_mesh_info_t": dfm.MeshInfo, "dfm_params": dfm.Params, "dfm_op_info_t": dfm.OpInfo,
               "dfm_solve_opts": dfm.SolveOpts, "dfm_solve_info": dfm.SolveInfo}
    for cname, py in mirrors.items():
        want = c_layout[cname]
        assert ctypes.sizeof(py) == want["sizeof"], cname
        names = [f[0] for f in py._fields_]
        assert sorted(names) == sorted(k for k in want if k != "sizeof"), cname
        for name in names:
            assert getattr(py, name).offset == want[name], (cname, name)
