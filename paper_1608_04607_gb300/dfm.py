"""Python binding of libdfm (include/dfm.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts numpy
arrays and torch CUDA tensors to the C ABI's plain pointers and sizes, owns
the library handles and raises DFMError on a non-zero status.  There is no
CPU fallback: if libdfm.so cannot be loaded, importing the library raises.
PyTorch provides device memory and the current CUDA stream only.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libdfm.so")

DFM_OK = 0
DFM_ERR_ARG = -1
DFM_ERR_MESH = -2
DFM_ERR_CUDA = -3
DFM_ERR_OOM = -4
DFM_ERR_NOT_CONVERGED = -5
DFM_ERR_NONFINITE = -6
DFM_ERR_UNSUPPORTED = -7
DFM_ERR_TIMEOUT = -8

F64, F32, BF16, F16, FP8E4M3 = 0, 1, 2, 3, 4
NEUMANN, GMRES, GMRES_IR = 0, 1, 2


class DFMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dfm error {code}: {msg}")
        self.code = code


class MeshInfo(ctypes.Structure):
    _fields_ = [("n_verts", ctypes.c_int64), ("n_tets", ctypes.c_int64), ("n_rows", ctypes.c_int64),
                ("n_boundary_rows", ctypes.c_int64), ("min_abs_volume", ctypes.c_double),
                ("total_volume", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("Np", ctypes.c_int), ("mu", ctypes.c_void_p), ("mu_uniform", ctypes.c_double),
                ("quad_order", ctypes.c_int), ("max_patch_deg", ctypes.c_double), ("precision", ctypes.c_int),
                ("moment", ctypes.c_int), ("c", ctypes.c_void_p), ("rho_f", ctypes.c_void_p)]


class OpInfo(ctypes.Structure):
    _fields_ = [("Np", ctypes.c_int), ("nb", ctypes.c_int), ("precision", ctypes.c_int), ("n_rows", ctypes.c_int64),
                ("row_stride", ctypes.c_int64), ("vals", ctypes.c_void_p), ("bytes", ctypes.c_int64)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("restart", ctypes.c_int), ("use_x0", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("transpose", ctypes.c_int), ("poly_degree", ctypes.c_int), ("precond_precision", ctypes.c_int),
                ("batch", ctypes.c_int), ("block", ctypes.c_int), ("coarse", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("resid", ctypes.c_double)]


_lib = None

# every entry point of include/dfm.h with its ctypes signature
_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "dfm_mesh_create": (_i, [_vp, _i64, _vp, _i64, _vp, _d, _vp, ctypes.POINTER(_vp)]),
    "dfm_mesh_destroy": (None, [_vp]),
    "dfm_mesh_info": (_i, [_vp, ctypes.POINTER(MeshInfo)]),
    "dfm_mesh_recv": (_i, [_vp, _vp]),
    "dfm_face_match_static": (_i, [_vp, _i64, _i64, _vp, ctypes.POINTER(ctypes.c_int64), _vp]),
    "dfm_gauss_legendre": (_i, [_i, _vp, _vp, _vp]),
    "dfm_assemble": (_i, [_vp, ctypes.POINTER(Params), _vp, ctypes.POINTER(_vp)]),
    "dfm_assemble_into": (_i, [_vp, ctypes.POINTER(Params), _vp, _vp]),
    "dfm_op_destroy": (None, [_vp]),
    "dfm_op_info": (_i, [_vp, ctypes.POINTER(OpInfo)]),
    "dfm_op_copy_vals": (_i, [_vp, _vp, _i64, _vp]),
    "dfm_op_copy_reflected": (_i, [_vp, _vp, _i64, _vp]),
    "dfm_apply": (_i, [_vp, _vp, _vp, _vp, _i, _d, _i, _i, _vp]),
    "dfm_source": (_i, [_vp, _i, _vp, _i, _vp, _vp]),
    "dfm_source_directed": (_i, [_vp, _i, _vp, _vp, _i, _i, _vp, _vp]),
    "dfm_point_source": (_i, [_vp, _i, _vp, _i, _vp, _d, _d, _i, _vp, _vp]),
    "dfm_apply_combo": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _i, _d, _i, _vp]),
    "dfm_precond_apply": (_i, [_vp, _i, _i, _i, _vp, _vp, _i, _vp]),
    "dfm_solve_combo": (_i, [_vp, _i, _vp, _vp, _i, _vp, ctypes.POINTER(SolveOpts), _vp, ctypes.POINTER(SolveInfo)]),
    "dfm_solve": (_i, [_vp, _vp, _i, _vp, ctypes.POINTER(SolveOpts), _vp, ctypes.POINTER(SolveInfo)]),
    "dfm_solve_damped": (_i, [_vp, _i, _vp, _vp, _i, _vp, ctypes.POINTER(SolveOpts), _vp,
                              ctypes.POINTER(SolveInfo)]),
    "dfm_op_check_error": (_i, [_vp, _vp]),
    "dfm_selftest_timeout": (_i, [_vp, _i, _vp]),
    "dfm_interior_density": (_i, [_vp, _i, _vp, _d, _vp, _vp, _i, _i, _vp, _vp, _vp]),
    "dfm_tet_density": (_i, [_vp, _i, _vp, _vp, _i, _vp, _vp]),
    "dfm_adjoint": (_i, [_vp, ctypes.POINTER(Params), _vp, _i, _vp, _vp, _vp, _vp, ctypes.POINTER(SolveOpts), _vp,
                         ctypes.POINTER(SolveInfo)]),
    "dfm_autotune": (_i, [_i]),
    "dfm_hop_graphs": (_i, [_i]),
    "dfm_hop_graph_replays": (ctypes.c_longlong, []),
    "dfm_autotune_report": (_i64, [ctypes.c_char_p, _i64]),
    "dfm_launch_count": (ctypes.c_longlong, []),
    "dfm_stats_enable": (_i, [_i]),
    "dfm_stats_reset": (_i, []),
    "dfm_kernel_stats": (_i, [_i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
    "dfm_op_nodes": (_i, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "dfm_last_error": (ctypes.c_char_p, []),
    "dfm_version": (ctypes.c_char_p, []),
}


def load(path: str = LIB_PATH):
    """Load libdfm.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        from . import build as _build

        _build.build()
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc, what=""):
    if rc != DFM_OK:
        msg = _lib.dfm_last_error().decode()
        raise DFMError(rc, f"{what}: {msg}" if what else msg)


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    """Device pointer of a contiguous torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _vec(t, rows, nb, dtypes, what):
    """Check a coefficient tensor [R, rows, nb] or [rows, nb] of an allowed dtype
    before its pointer crosses the ABI (the library cannot see sizes); returns R."""
    import torch

    if not isinstance(t, torch.Tensor) or t.dtype not in dtypes or t.dim() not in (2, 3) \
            or tuple(t.shape[-2:]) != (rows, nb):
        got = (tuple(t.shape), t.dtype) if isinstance(t, torch.Tensor) else type(t).__name__
        raise DFMError(DFM_ERR_ARG, f"{what}: expected [R, {rows}, {nb}] or [{rows}, {nb}] of "
                                    f"{'/'.join(str(d) for d in dtypes)}, got {got}")
    return 1 if t.dim() == 2 else t.shape[0]


def _like(t, ref, what):
    """Check that an optional companion tensor has ref's dtype and shape."""
    import torch

    if t is not None and (not isinstance(t, torch.Tensor) or t.dtype != ref.dtype or t.shape != ref.shape):
        raise DFMError(DFM_ERR_ARG, f"{what}: expected {tuple(ref.shape)} {ref.dtype}")


def basis(Np: int, spatial: int = 0) -> int:
    """Basis code of the C ABI (DFM_BASIS): momentum order Np with the
    piecewise-constant spatial function per face (spatial=0, Sec. 3.1) or the
    linear spatial basis, three orthonormal affine functions per face
    (spatial=1).  Every argument named Np accepts a code."""
    return int(Np) | (int(spatial) << 8)


def nbasis(Np: int) -> int:
    """Unknowns per row of basis code Np: (Np+1)(Np+2)/2 per spatial function."""
    n = Np & 0xFF
    return (3 if Np >> 8 else 1) * ((n + 1) * (n + 2) // 2)


class Mesh:
    """A tetrahedral mesh on the device (dfm_mesh_create)."""

    def __init__(self, verts, tets, refl=0.95):
        L = load()
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tets, dtype=np.int32)
        if np.ndim(refl) == 0:
            rp, rd = None, float(refl)
        else:
            r = np.ascontiguousarray(refl, dtype=np.float64)
            rp, rd = r.ctypes.data_as(ctypes.c_void_p), 0.0
        h = ctypes.c_void_p()
        _check(L.dfm_mesh_create(v.ctypes.data_as(ctypes.c_void_p), v.shape[0], t.ctypes.data_as(ctypes.c_void_p),
                                 t.shape[0], rp, rd, _stream(), ctypes.byref(h)), "dfm_mesh_create")
        self._h = h
        self.n_tets = int(t.shape[0])
        self.n_rows = 4 * self.n_tets

    @property
    def handle(self):
        return self._h

    def info(self) -> MeshInfo:
        mi = MeshInfo()
        _check(_lib.dfm_mesh_info(self._h, ctypes.byref(mi)), "dfm_mesh_info")
        return mi

    def recv(self) -> np.ndarray:
        out = np.empty(self.n_rows, dtype=np.int32)
        _check(_lib.dfm_mesh_recv(self._h, out.ctypes.data_as(ctypes.c_void_p)), "dfm_mesh_recv")
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.dfm_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """The assembled operator B (dfm_assemble)."""

    def __init__(self, mesh: Mesh, Np: int, mu=0.0, precision=F32, quad_order=0, max_patch_deg=0.0, moment=0,
                 c=None, rho_f=None):
        """c, rho_f: per-tet propagation speed and fluid density (heterogeneous
        media, Sec. 3.3), tensors or arrays of n_tets values, or None (1)."""
        import torch

        self.mesh = mesh
        self._keep = []
        self.moment = moment
        self._media = []
        for v, what in ((c, "c"), (rho_f, "rho_f")):
            if v is None:
                self._media.append(None)
                continue
            t = torch.as_tensor(v, dtype=torch.float64, device="cuda").contiguous().reshape(-1)
            if t.numel() != mesh.n_tets:
                raise DFMError(DFM_ERR_ARG, f"{what}: expected {mesh.n_tets} per-tet values")
            self._media.append(t)
        p = self._params(Np, mu, precision, quad_order, max_patch_deg)
        self._p = p
        h = ctypes.c_void_p()
        _check(_lib.dfm_assemble(mesh.handle, ctypes.byref(p), _stream(), ctypes.byref(h)), "dfm_assemble")
        self._h = h
        oi = OpInfo()
        _check(_lib.dfm_op_info(h, ctypes.byref(oi)), "dfm_op_info")
        self.Np, self.nb, self.precision = oi.Np, oi.nb, oi.precision
        self.n_rows, self.row_stride, self.bytes = oi.n_rows, oi.row_stride, oi.bytes
        self._torch = torch

    def _params(self, Np, mu, precision, quad_order, max_patch_deg):
        import torch

        p = Params()
        p.Np = Np
        if isinstance(mu, torch.Tensor) and mu.dim() == 0:
            mu = float(mu)
        if isinstance(mu, torch.Tensor):
            # the library reads n_tets values through the pointer
            if mu.numel() != self.mesh.n_tets:
                raise DFMError(DFM_ERR_ARG, f"mu: expected {self.mesh.n_tets} per-tet values, got shape "
                                            f"{tuple(mu.shape)}")
            mu_t = mu.to(device="cuda", dtype=torch.float64).contiguous().reshape(-1)
            self._keep = [mu_t]
            p.mu = mu_t.data_ptr()
            p.mu_uniform = 0.0
        else:
            p.mu = None
            p.mu_uniform = float(mu)
        p.quad_order = quad_order
        p.max_patch_deg = max_patch_deg
        p.precision = precision
        p.moment = getattr(self, "moment", 0)
        media = getattr(self, "_media", [None, None])
        p.c = media[0].data_ptr() if media[0] is not None else None
        p.rho_f = media[1].data_ptr() if media[1] is not None else None
        return p

    def reassemble(self, mu, quad_order=0, max_patch_deg=0.0):
        p = self._params(self.Np, mu, self.precision, quad_order, max_patch_deg)
        self._p = p
        _check(_lib.dfm_assemble_into(self.mesh.handle, ctypes.byref(p), self._h, _stream()), "dfm_assemble_into")

    @property
    def handle(self):
        return self._h

    def check_error(self):
        """Raise DFMError(DFM_ERR_TIMEOUT) if a kernel of this operator gave up
        waiting for its data since the last check (dfm_op_check_error)."""
        _check(_lib.dfm_op_check_error(self._h, _stream()), "dfm_op_check_error")

    def blocks(self):
        """Copy of the block storage as a torch CUDA tensor [rows, 3, nb, nb]."""
        torch = self._torch
        dt = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16}[self.precision]
        buf = torch.empty(self.n_rows * self.row_stride, dtype=dt, device="cuda")
        _check(_lib.dfm_op_copy_vals(self._h, _ptr(buf), self.bytes, _stream()), "dfm_op_copy_vals")
        nb = self.nb
        return buf.view(self.n_rows, self.row_stride)[:, :3 * nb * nb].reshape(self.n_rows, 3, nb, nb)

    def blocks_reflected(self):
        """The reflected part (heterogeneous media) as [rows, 3, nb, nb]: row
        R = 4t + l' holds the blocks reflected at face l' from tet t's other faces."""
        torch = self._torch
        dt = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16}[self.precision]
        buf = torch.empty(self.n_rows * self.row_stride, dtype=dt, device="cuda")
        _check(_lib.dfm_op_copy_reflected(self._h, _ptr(buf), self.bytes, _stream()), "dfm_op_copy_reflected")
        nb = self.nb
        return buf.view(self.n_rows, self.row_stride)[:, :3 * nb * nb].reshape(self.n_rows, 3, nb, nb)

    def apply(self, x, x0=None, alpha=1.0, trans=False, out=None):
        """y = x0 + alpha B x (or B^T x); x of shape [R, rows, nb] or [rows, nb]."""
        torch = self._torch
        R = _vec(x, self.n_rows, self.nb, (torch.float32, torch.float64), "apply: x")
        _like(x0, x, "apply: x0")
        _like(out, x, "apply: out")
        xtype = {torch.float64: F64, torch.float32: F32}[x.dtype]
        y = torch.empty_like(x) if out is None else out
        _check(_lib.dfm_apply(self._h, _ptr(x), _ptr(x0), _ptr(y), R, float(alpha), int(bool(trans)), xtype,
                              _stream()), "dfm_apply")
        return y

    def precond(self, x, degree=16, precision=F16, out=None, transpose=False):
        """z = sum_{k<degree} B~^k x on the low-precision copy B~ of the blocks
        (dfm_precond_apply; precision F16, BF16 or FP8E4M3); x: FP32
        [R, rows, nb] or [rows, nb]."""
        torch = self._torch
        if x.dtype != torch.float32:
            raise TypeError("precond: x must be float32")
        R = _vec(x, self.n_rows, self.nb, (torch.float32,), "precond: x")
        _like(out, x, "precond: out")
        z = torch.empty_like(x) if out is None else out
        _check(_lib.dfm_precond_apply(self._h, int(precision), int(degree), int(bool(transpose)), _ptr(x), _ptr(z), R,
                                      _stream()), "dfm_precond_apply")
        return z

    def solve(self, rho0, method=GMRES_IR, tol=1e-8, max_iter=0, restart=0, x0=None, inner_tol=0.0,
              raise_on_nonconvergence=True, transpose=False, poly_degree=0, batch=0, precond_precision=0, block=0,
              coarse=0):
        """rho = (I - B)^{-1} rho0 (FP64, [R, rows, nb] or [rows, nb]); returns (rho, SolveInfo).
        block=1: groups of right-hand sides share one Krylov space (dfm_solve_opts.block);
        coarse=g: two-level preconditioner on g^3 aggregates (dfm_solve_opts.coarse)."""
        torch = self._torch
        R = _vec(rho0, self.n_rows, self.nb, (torch.float64,), "solve: rho0")
        _like(x0, rho0, "solve: x0")
        rho = torch.empty_like(rho0) if x0 is None else x0.clone()
        o = SolveOpts(method=method, tol=tol, max_iter=max_iter, restart=restart, use_x0=int(x0 is not None),
                      inner_tol=inner_tol, transpose=int(bool(transpose)), poly_degree=poly_degree,
                      precond_precision=precond_precision, batch=batch, block=int(bool(block)), coarse=int(coarse))
        info = SolveInfo()
        rc = _lib.dfm_solve(self._h, _ptr(rho0), R, _ptr(rho), ctypes.byref(o), _stream(), ctypes.byref(info))
        if rc == DFM_ERR_NOT_CONVERGED and not raise_on_nonconvergence:
            return rho, info
        _check(rc, "dfm_solve")
        return rho, info

    def adjoint(self, rho, gvec, dgvec=None, method=GMRES_IR, tol=1e-8, max_iter=0, restart=0, inner_tol=0.0,
                poly_degree=0, precond_precision=0, lam0=None):
        """lambda = (I - B)^{-T} gvec and dJ/dmu for J = sum_r gvec . rho_r (dfm_adjoint).
        rho: FP64 [R, rows, nb]; gvec/dgvec: FP64 [rows, nb]; lam0: initial guess
        for lambda (e.g. an earlier call's lambda for the same operator and
        functional).  Returns (lambda, dJ_dmu [R, n_tets], info)."""
        torch = self._torch
        R = _vec(rho, self.n_rows, self.nb, (torch.float64,), "adjoint: rho")
        if _vec(gvec, self.n_rows, self.nb, (torch.float64,), "adjoint: gvec") != 1 or gvec.dim() != 2:
            raise DFMError(DFM_ERR_ARG, "adjoint: gvec must be [rows, nb]")
        _like(dgvec, gvec, "adjoint: dgvec")
        _like(lam0, gvec, "adjoint: lam0")
        lam = (torch.empty((self.n_rows, self.nb), dtype=torch.float64, device="cuda") if lam0 is None
               else lam0.clone())
        dj = torch.empty((R, self.mesh.n_tets), dtype=torch.float64, device="cuda")
        o = SolveOpts(method=method, tol=tol, max_iter=max_iter, restart=restart, use_x0=int(lam0 is not None),
                      inner_tol=inner_tol,
                      transpose=1, poly_degree=poly_degree, batch=0, precond_precision=precond_precision)
        info = SolveInfo()
        _check(_lib.dfm_adjoint(self._h, ctypes.byref(self._p), _ptr(rho), R, _ptr(gvec), _ptr(dgvec), _ptr(lam),
                                _ptr(dj), ctypes.byref(o), _stream(), ctypes.byref(info)), "dfm_adjoint")
        return lam, dj, info

    def close(self):
        if getattr(self, "_h", None):
            _lib.dfm_op_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def source(mesh: Mesh, Np: int, rows):
    """Unit isotropic sources on the given rows: FP64 [n_src, rows, nb] (dfm_source)."""
    import torch

    rows = np.ascontiguousarray(np.atleast_1d(rows), dtype=np.int64)
    out = torch.empty((rows.size, mesh.n_rows, nbasis(Np)), dtype=torch.float64, device="cuda")
    _check(_lib.dfm_source(mesh.handle, Np, rows.ctypes.data_as(ctypes.c_void_p), rows.size, _ptr(out), _stream()),
           "dfm_source")
    return out


def source_directed(mesh: Mesh, Np: int, rows, dirs=None, combine=False):
    """Unit densities along one ray direction per row (dfm_source_directed):
    dirs [n_src, 3] (None = each row's inward normal, Eq. RhoNeumann).  Returns
    FP64 [n_src, rows, nb], or [rows, nb] with every source in one right-hand
    side when combine is set."""
    import torch

    rows = np.ascontiguousarray(np.atleast_1d(rows), dtype=np.int64)
    dp = None
    if dirs is not None:
        d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(rows.size, 3))
        dp = d.ctypes.data_as(ctypes.c_void_p)
    shape = (mesh.n_rows, nbasis(Np)) if combine else (rows.size, mesh.n_rows, nbasis(Np))
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    _check(load().dfm_source_directed(mesh.handle, Np, rows.ctypes.data_as(ctypes.c_void_p), dp, rows.size,
                                      int(bool(combine)), _ptr(out), _stream()), "dfm_source_directed")
    return out


def point_source(mesh: Mesh, Np: int, r0, mu=0.0, strength=1.0, nq=0):
    """Point sources at r0 [n_src, 3] (or one [3]) in uniform media
    (dfm_point_source, Eq. SourceRho): FP64 [n_src, rows, nb].  mu: a float or
    a per-tet tensor; nq = 0: the split polar rule with 24 points per
    direction, nq < 0: that rule with |nq| points, nq > 0: the collapsed Gauss
    rule of that order."""
    import torch

    r0 = np.ascontiguousarray(np.asarray(r0, dtype=np.float64).reshape(-1, 3))
    out = torch.empty((r0.shape[0], mesh.n_rows, nbasis(Np)), dtype=torch.float64, device="cuda")
    keep = None
    if isinstance(mu, torch.Tensor):
        keep = mu.to(device="cuda", dtype=torch.float64).contiguous()
        if keep.numel() != mesh.n_tets:
            raise DFMError(DFM_ERR_ARG, "point_source: mu must hold one value per tet")
        mup, muu = _ptr(keep), 0.0
    else:
        mup, muu = None, float(mu)
    _check(load().dfm_point_source(mesh.handle, Np, r0.ctypes.data_as(ctypes.c_void_p), r0.shape[0], mup, muu,
                                   float(strength), int(nq), _ptr(out), _stream()), "dfm_point_source")
    return out


def _op_array(ops):
    arr = (ctypes.c_void_p * len(ops))(*[o.handle.value for o in ops])
    return arr


def apply_combo(ops, coef, x, x0=None, alpha=1.0, out=None):
    """y_r = x0_r + alpha sum_k coef[r, k] B_k x_r (dfm_apply_combo); x FP32/FP64 [R, rows, nb]."""
    import torch

    coef = np.ascontiguousarray(coef, dtype=np.float64)
    R = _vec(x, ops[0].n_rows, ops[0].nb, (torch.float32, torch.float64), "apply_combo: x")
    _like(x0, x, "apply_combo: x0")
    _like(out, x, "apply_combo: out")
    if coef.shape != (R, len(ops)):
        raise DFMError(DFM_ERR_ARG, f"apply_combo: coef must be [{R}, {len(ops)}]")
    xtype = {torch.float64: F64, torch.float32: F32}[x.dtype]
    y = torch.empty_like(x) if out is None else out
    _check(load().dfm_apply_combo(_op_array(ops), len(ops), coef.ctypes.data_as(ctypes.c_void_p), _ptr(x), _ptr(x0),
                                  _ptr(y), R, float(alpha), xtype, _stream()), "dfm_apply_combo")
    return y


def solve_combo(ops, coef, rho0, tol=1e-8, max_iter=0, restart=0, inner_tol=0.0, poly_degree=0, batch=0,
                precond_precision=0):
    """rho_r = (I - sum_k coef[r, k] B_k)^{-1} rho0_r (dfm_solve_combo); returns (rho, SolveInfo)."""
    import torch

    coef = np.ascontiguousarray(coef, dtype=np.float64)
    R = _vec(rho0, ops[0].n_rows, ops[0].nb, (torch.float64,), "solve_combo: rho0")
    if coef.shape != (R, len(ops)):
        raise DFMError(DFM_ERR_ARG, f"solve_combo: coef must be [{R}, {len(ops)}]")
    rho = torch.empty_like(rho0)
    o = SolveOpts(method=GMRES_IR, tol=tol, max_iter=max_iter, restart=restart, use_x0=0, inner_tol=inner_tol,
                  transpose=0, poly_degree=poly_degree, batch=batch, precond_precision=precond_precision)
    info = SolveInfo()
    _check(load().dfm_solve_combo(_op_array(ops), len(ops), coef.ctypes.data_as(ctypes.c_void_p), _ptr(rho0), R,
                                  _ptr(rho), ctypes.byref(o), _stream(), ctypes.byref(info)), "dfm_solve_combo")
    return rho, info


def solve_damped(moments, mu_rhs, rho0, tol=1e-8, max_iter=0, restart=0, inner_tol=0.0, poly_degree=0, batch=0,
                 precond_precision=0):
    """rho_r = (I - B(mu_r))^{-1} rho0_r for per-right-hand-side uniform damping
    mu_r, from the damping moments moments[k] (Operator(..., moment=k), all at
    one uniform mu_c); the library forms B(mu_r) = sum_k (mu_r - mu_c)^k / k!
    B^(k) (dfm_solve_damped).  Returns (rho, SolveInfo)."""
    import torch

    mu = np.ascontiguousarray(np.atleast_1d(mu_rhs), dtype=np.float64)
    R = _vec(rho0, moments[0].n_rows, moments[0].nb, (torch.float64,), "solve_damped: rho0")
    if mu.shape != (R,):
        raise DFMError(DFM_ERR_ARG, f"solve_damped: mu_rhs must hold {R} values")
    rho = torch.empty_like(rho0)
    o = SolveOpts(method=GMRES_IR, tol=tol, max_iter=max_iter, restart=restart, use_x0=0, inner_tol=inner_tol,
                  transpose=0, poly_degree=poly_degree, batch=batch, precond_precision=precond_precision)
    info = SolveInfo()
    _check(load().dfm_solve_damped(_op_array(moments), len(moments), mu.ctypes.data_as(ctypes.c_void_p), _ptr(rho0),
                                   R, _ptr(rho), ctypes.byref(o), _stream(), ctypes.byref(info)), "dfm_solve_damped")
    return rho, info


def selftest_timeout(op, polls=1000):
    """Run the library's time-out self-test kernel on op (dfm_selftest_timeout):
    a bounded wait that nothing completes sets op's time-out flag."""
    _check(load().dfm_selftest_timeout(op.handle, int(polls), _stream()), "dfm_selftest_timeout")


def interior_density(mesh: Mesh, Np: int, tets, weights=None, mu=0.0, nq=0, gvec=None, dgvec=None):
    """Interior density coefficients at tet centroids (dfm_interior_density):
    adds w_e g_e into gvec and w_e dg_e/dmu_e into dgvec (FP64 [rows, nb], created
    zeroed when not given).  J(rho) = (gvec * rho).sum().  nq = 0 (default):
    the split polar rule with 24 points per direction; nq < 0: that rule with
    |nq| points (both accurate for thin tets); nq > 0: the flat collapsed Gauss
    rule of that order per face."""
    import torch

    nb = nbasis(Np)
    tets = np.ascontiguousarray(np.atleast_1d(tets), dtype=np.int64)
    if gvec is None:
        gvec = torch.zeros((mesh.n_rows, nb), dtype=torch.float64, device="cuda")
    if dgvec is None:
        dgvec = torch.zeros((mesh.n_rows, nb), dtype=torch.float64, device="cuda")
    for t, what in ((gvec, "interior_density: gvec"), (dgvec, "interior_density: dgvec")):
        if _vec(t, mesh.n_rows, nb, (torch.float64,), what) != 1 or t.dim() != 2:
            raise DFMError(DFM_ERR_ARG, f"{what} must be [rows, nb]")
    wp = None
    if weights is not None:
        w = np.ascontiguousarray(np.broadcast_to(np.asarray(weights, dtype=np.float64), tets.shape))
        wp = w.ctypes.data_as(ctypes.c_void_p)
    keep = None
    if isinstance(mu, torch.Tensor):
        keep = mu.to(device="cuda", dtype=torch.float64).contiguous()
        mup, muu = _ptr(keep), 0.0
    else:
        mup, muu = None, float(mu)
    _check(load().dfm_interior_density(mesh.handle, Np, mup, muu, tets.ctypes.data_as(ctypes.c_void_p), wp,
                                       tets.size, nq, _ptr(gvec), _ptr(dgvec), _stream()), "dfm_interior_density")
    return gvec, dgvec


def tet_density(mesh: Mesh, Np: int, gvec, rho):
    """Per-tet sums of gvec . rho over each tet's four rows (dfm_tet_density):
    rho FP64 [R, rows, nb] or [rows, nb]; returns FP64 [R, n_tets] or [n_tets].
    With gvec from interior_density over all tets this is rho_T at every centroid."""
    import torch

    nb = nbasis(Np)
    R = _vec(rho, mesh.n_rows, nb, (torch.float64,), "tet_density: rho")
    if _vec(gvec, mesh.n_rows, nb, (torch.float64,), "tet_density: gvec") != 1 or gvec.dim() != 2:
        raise DFMError(DFM_ERR_ARG, "tet_density: gvec must be [rows, nb]")
    out = torch.empty((R, mesh.n_tets), dtype=torch.float64, device="cuda")
    _check(load().dfm_tet_density(mesh.handle, Np, _ptr(gvec), _ptr(rho), R, _ptr(out), _stream()),
           "dfm_tet_density")
    return out[0] if rho.dim() == 2 else out


class DFMSolve:
    """rho = (I - B(mu))^{-1} rho0 as a torch.autograd.Function of the per-tet
    damping mu: forward = dfm_assemble + dfm_solve, backward = dfm_adjoint
    (grad_mu = lambda^T dB/dmu rho, grad_rho0 = lambda).  A functional with
    its own explicit mu-dependence (the dgvec of interior_density) adds
    dgvec . rho per tet itself.  mu: per-tet [n_tets] tensor, or a 0-dim tensor
    for uniform damping (its gradient is then the sum over tets)."""

    @staticmethod
    def apply(mesh, Np, mu, rho0, tol=1e-8, **solve_kw):
        import torch

        def _grad_mu(per_tet):
            # a scalar (uniform) damping moves every tet's mu together
            if mu.dim() == 0:
                return per_tet.sum().to(mu.dtype)
            return per_tet.reshape(mu.shape).to(mu.dtype)

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, mu_t, rho0_t):
                op = Operator(mesh, Np, mu=mu_t.detach(), precision=F32)
                rho, _ = op.solve(rho0_t.detach().contiguous(), tol=tol, **solve_kw)
                ctx.op = op
                ctx.save_for_backward(rho)
                return rho

            @staticmethod
            def backward(ctx, grad_rho):
                (rho,) = ctx.saved_tensors
                op = ctx.op
                g = grad_rho.contiguous()
                R = 1 if rho.dim() == 2 else rho.shape[0]
                gsum = g if g.dim() == 2 else g
                if gsum.dim() == 3 and gsum.shape[0] > 1:
                    # one adjoint solve per distinct functional
                    grads, lams = [], []
                    for r in range(gsum.shape[0]):
                        lam, dj, _ = op.adjoint(rho[r:r + 1], gsum[r], tol=tol)
                        grads.append(dj[0])
                        lams.append(lam)
                    return _grad_mu(torch.stack(grads).sum(0)), torch.stack(lams)
                lam, dj, _ = op.adjoint(rho, gsum.reshape(op.n_rows, op.nb), tol=tol)
                return _grad_mu(dj.sum(0)), lam.reshape(rho0.shape)

        return _Fn.apply(mu, rho0)


def gauss_legendre(q: int):
    """Gauss-Legendre nodes/weights computed on the device (dfm_gauss_legendre)."""
    import torch

    x = torch.empty(q, dtype=torch.float64, device="cuda")
    w = torch.empty(q, dtype=torch.float64, device="cuda")
    load()
    _check(_lib.dfm_gauss_legendre(q, _ptr(x), _ptr(w), _stream()), "dfm_gauss_legendre")
    return x, w


(KERNEL_ASSEMBLE, KERNEL_SPMV, KERNEL_SPMV_T, KERNEL_DOT, KERNEL_AXPY, KERNEL_SPMV64, KERNEL_CONTRACT, KERNEL_SPMV16,
 KERNEL_SPMV16_T, KERNEL_SPMV64_T) = range(10)


def autotune(mode: int = 1):
    """0: fixed default launch geometries; 1: tune on first use (default);
    2: forget the tuned choices and tune again (dfm_autotune)."""
    _check(load().dfm_autotune(int(mode)), "dfm_autotune")


def hop_graphs(mode: int = -1) -> bool:
    """CUDA graphs of the preconditioner's Horner chains (dfm_hop_graphs):
    1 on (default), 0 off, -1 query; returns the state after the call."""
    rc = load().dfm_hop_graphs(int(mode))
    if rc < 0:
        _check(rc, "dfm_hop_graphs")
    return bool(rc)


def hop_graph_replays() -> int:
    """Hop-chain graph replays so far (dfm_hop_graph_replays)."""
    return int(load().dfm_hop_graph_replays())


def autotune_report() -> list:
    """The autotuner's choices per launch shape (dfm_autotune_report)."""
    import json

    L = load()
    n = int(L.dfm_autotune_report(None, 0))
    buf = ctypes.create_string_buffer(n)
    L.dfm_autotune_report(buf, n)
    return json.loads(buf.value.decode())


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().dfm_launch_count())


def stats_enable(on=True):
    """True or 1: time every launch of the timed kernels; n > 1: every n-th
    launch of each kernel; False or 0: stop (dfm_stats_enable)."""
    _check(load().dfm_stats_enable(int(on)), "dfm_stats_enable")


def stats_reset():
    _check(load().dfm_stats_reset(), "dfm_stats_reset")


def kernel_stats(kernel: int):
    """(launches, total device ms) of one kernel since the last reset."""
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    _check(load().dfm_kernel_stats(kernel, ctypes.byref(n), ctypes.byref(ms)), "dfm_kernel_stats")
    return int(n.value), float(ms.value)


def op_nodes(op: "Operator") -> int:
    n = ctypes.c_int64()
    _check(load().dfm_op_nodes(op.handle, ctypes.byref(n)), "dfm_op_nodes")
    return int(n.value)


def version() -> str:
    return load().dfm_version().decode()
