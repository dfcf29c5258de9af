"""The allocation-free face matching entry point (dfm_face_match_static).

Some callers cannot call cudaMalloc (their device memory is reserved by their
own pool, or they must not enter the CUDA allocator where they run); this
entry point keeps its hash table in a fixed device array instead.  The test
calls it through the C ABI twice in a row, on two different meshes, and checks
each result against the allocating entry point (dfm_mesh_create): the face
matching is integer work, so the comparison is exact.  It also checks that an
oversized mesh is rejected before any GPU work.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import need_gpu
from paper_1608_04607_gb300.inputs import kuhn_cube_mesh

pytestmark = pytest.mark.gpu


def _call(dfm, lib, tets_np, n_verts):
    import torch

    tets_d = torch.tensor(tets_np, dtype=torch.int32, device="cuda").contiguous()
    recv_d = torch.full((4 * tets_np.shape[0],), -7, dtype=torch.int32, device="cuda")
    nb = ctypes.c_int64(-1)
    rc = lib.dfm_face_match_static(ctypes.c_void_p(tets_d.data_ptr()), n_verts, tets_np.shape[0],
                                   ctypes.c_void_p(recv_d.data_ptr()), ctypes.byref(nb),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, recv_d.cpu().numpy(), nb.value


def test_static_face_matching_matches_allocating_path():
    need_gpu()
    from paper_1608_04607_gb300 import dfm

    lib = dfm.load()
    # first a larger mesh, then a smaller one: stale table entries from the
    # first call would corrupt the second if the table were not re-initialised
    for n, seed in ((7, 3), (3, 5)):
        m = kuhn_cube_mesh(n, jitter=0.2, seed=seed)
        mesh = dfm.Mesh(m.verts, m.tets, refl=0.9)
        ref = mesh.recv()
        rc, got, nb = _call(dfm, lib, m.tets, m.verts.shape[0])
        assert rc == dfm.DFM_OK, lib.dfm_last_error().decode()
        np.testing.assert_array_equal(got, ref)
        assert nb == mesh.info().n_boundary_rows == 12 * n * n


def test_static_face_matching_rejects_oversized_mesh():
    need_gpu()
    from paper_1608_04607_gb300 import dfm

    lib = dfm.load()
    n_tets = 131072 + 1
    rc = lib.dfm_face_match_static(ctypes.c_void_p(16), 10, n_tets, ctypes.c_void_p(16), None, None)
    assert rc == dfm.DFM_ERR_ARG
    assert "131072" in lib.dfm_last_error().decode()
