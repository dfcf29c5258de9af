"""Python side of the FP64 CPU oracle for discrete flow mapping.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product (the CUDA library and its
binding) never imports this module, and this module imports nothing from the
product except the seeded input generators, which hold no method arithmetic.

The quadrature-heavy parts live in dfm_oracle.c (loaded through ctypes); this
file does the orchestration in plain numpy: mesh topology by a dictionary of
sorted vertex triples, the Galerkin source vector, operator application,
direct and Krylov solves, the interior density functional and the adjoint
gradient.  Each function names the part of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dfm_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile dfm_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_blocks.restype = ctypes.c_int
        L.orc_mc_block.restype = ctypes.c_int
        L.orc_blocks_p1.restype = ctypes.c_int
        L.orc_mc_block_p1.restype = ctypes.c_int
        L.orc_region_cos_measure.restype = ctypes.c_double
        L.orc_transmission.restype = ctypes.c_double
        L.orc_transmission.argtypes = [ctypes.c_double] * 4
        _lib = L
    return _lib


def _p(a, typ=_dp):
    return a.ctypes.data_as(typ)


def nbasis(Np: int) -> int:
    """Number of momentum basis functions for order Np (Sec. 3.1, Eq. FBApprox)."""
    return (Np + 1) * (Np + 2) // 2


def zernike_index(n: int, m: int) -> int:
    return (n * (n + 2) + m) // 2


def zernike_nm(Np: int):
    """(n, m) of each basis index, in index order."""
    out = []
    for n in range(Np + 1):
        for m in range(-n, n + 1, 2):
            out.append((n, m))
    return out


def zernike(Np: int, px, py) -> np.ndarray:
    """Zernike polynomials Z_n^m at points p of the unit disc (Sec. 3.1), [npts, nb]."""
    px = np.ascontiguousarray(np.atleast_1d(px), dtype=np.float64)
    py = np.ascontiguousarray(np.atleast_1d(py), dtype=np.float64)
    out = np.empty((px.size, nbasis(Np)), dtype=np.float64)
    lib().orc_zernike(ctypes.c_int(Np), ctypes.c_int64(px.size), _p(px), _p(py), _p(out))
    return out


def zernike_invnorm(Np: int) -> np.ndarray:
    """N_{nm} = (2n+2)/(eps_m pi), eps_0 = 2 (Sec. 3.1-3.2)."""
    return np.array([(2 * n + 2) / ((2.0 if m == 0 else 1.0) * np.pi) for n, m in zernike_nm(Np)])


# Gauss-Legendre orders used by the oracle; the direction integral doubles
# through these, the spatial (triangle) integral uses TRI_ORDER.
GL_ORDERS = (4, 8, 16, 32, 64)
TRI_ORDER = 12


class _GL:
    def __init__(self, orders):
        xs, ws, offs = [], [], []
        off = 0
        for q in orders:
            x, w = np.polynomial.legendre.leggauss(q)
            xs.append(x)
            ws.append(w)
            offs.append(off)
            off += q
        self.qs = np.array(orders, dtype=np.int32)
        self.offs = np.array(offs, dtype=np.int32)
        self.x = np.concatenate(xs)
        self.w = np.concatenate(ws)


_gl_cache = {}


def gl_table(orders=GL_ORDERS + (TRI_ORDER,)):
    key = tuple(orders)
    if key not in _gl_cache:
        _gl_cache[key] = _GL(key)
    return _gl_cache[key]


# ---------------------------------------------------------------------------
# Mesh topology and face geometry
# ---------------------------------------------------------------------------

@dataclass
class Topology:
    """recv[4t + f] = the row that receives flux leaving tet t through face f:
    the neighbour's row across f, or 4t + f itself on the boundary.
    boundary[row] = True for boundary rows.  src_tet[R], src_face[R]: the tet
    whose flux row R receives and that tet's exit face (the inverse map)."""

    recv: np.ndarray
    boundary: np.ndarray
    src_tet: np.ndarray
    src_face: np.ndarray


def topology(tets: np.ndarray) -> Topology:
    """Face adjacency of a conforming tet mesh (Sec. 2) by a dictionary of sorted
    vertex triples.  Face f of tet t is the face opposite its local vertex f."""
    nt = tets.shape[0]
    seen = {}
    recv = np.arange(4 * nt, dtype=np.int64)
    for t in range(nt):
        tv = tets[t]
        for f in range(4):
            key = tuple(sorted(int(tv[k]) for k in range(4) if k != f))
            row = 4 * t + f
            if key in seen:
                other = seen.pop(key)
                recv[row] = other
                recv[other] = row
            else:
                seen[key] = row
    boundary = recv == np.arange(4 * nt)
    # row R receives from the tet on the other side (itself on the boundary)
    src_tet = recv // 4
    src_face = recv % 4
    return Topology(recv=recv, boundary=boundary, src_tet=src_tet, src_face=src_face)


def face_areas(verts: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """|T_{t,f}| for every row 4t + f."""
    out = np.empty(4 * tets.shape[0])
    for f in range(4):
        idx = [(f + 1 + k) % 4 for k in range(3)]
        a, b, c = (verts[tets[:, i]] for i in idx)
        out[f::4] = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    return out


# ---------------------------------------------------------------------------
# Operator blocks (Sec. 3.2-3.4)
# ---------------------------------------------------------------------------

@dataclass
class Operator:
    """Discretised transfer operator in the oracle's own column layout:
    blocks[J, k] (nb x nb, rows = test index on the receiving face, columns =
    trial index on the source face) for source column J = 4t + f and its k-th
    destination face fp != f (ascending), received by dest[J, k].
    dblocks: d(blocks)/d(mu_t) when requested.  q_used: accepted order."""

    Np: int
    blocks: np.ndarray
    dest: np.ndarray
    dblocks: np.ndarray | None = None
    q_used: np.ndarray | None = None
    # heterogeneous media (Sec. 3.3): rblocks[J, k] is the part of the flux of
    # column J that an interface between unequal media reflects back into the
    # column's own tet, received by rdest[J, k] = 4t + fp (zero blocks on the
    # boundary, where blocks already hold the reflection)
    rblocks: np.ndarray | None = None
    rdest: np.ndarray | None = None
    drblocks: np.ndarray | None = None
    # spatial functions per face: 1 (piecewise constant, Sec. 3.1) or 3 (the
    # linear basis); unknowns of a row are ordered s * nbasis(Np) + Zernike idx
    ns: int = 1

    @property
    def nb(self):
        return self.ns * nbasis(self.Np)

    @property
    def nrows(self):
        return self.blocks.shape[0]


def pair_list(nt: int):
    """All (t, f, fp) face pairs with fp != f, in column-major order."""
    t = np.repeat(np.arange(nt, dtype=np.int64), 12)
    f = np.tile(np.repeat(np.arange(4, dtype=np.int32), 3), nt)
    fp_tab = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]], dtype=np.int32)
    fp = np.tile(fp_tab.reshape(-1), nt)
    return t, f, fp


def blocks_for_pairs(verts, tets, topo: Topology, mu_tet, refl_row, Np, t, f, fp, q=None, rtol=1e-13,
                     lev0=1, with_derivative=False, regions_mask=0x0F, nthreads=0, spatial=0):
    """Blocks for the listed face pairs (t, f) -> fp.

    Fixed order when q is given (one of GL_ORDERS); otherwise the order doubles
    from GL_ORDERS[lev0] until the block max-norm changes by <= rtol relative.
    lambda = refl_row[recv] on boundary rows, 1 on interior faces (uniform media,
    transmission probability 1, Sec. 3.3).  The damping is mu of tet t.
    spatial=1: the linear spatial basis (3 orthonormal functions per face:
    Gram-Schmidt of 1, l_1, l_2 in the face's barycentric coordinates), blocks
    of side 3 nb.
    """
    G = gl_table()
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    t = np.ascontiguousarray(t, dtype=np.int64)
    f = np.ascontiguousarray(f, dtype=np.int32)
    fp = np.ascontiguousarray(fp, dtype=np.int32)
    n = t.size
    recv = np.ascontiguousarray(topo.recv[4 * t + fp], dtype=np.int64)
    mu = np.ascontiguousarray(np.asarray(mu_tet, dtype=np.float64)[t])
    refl_row = np.broadcast_to(np.asarray(refl_row, dtype=np.float64), (4 * tets.shape[0],))
    lam = np.where(topo.boundary[recv], refl_row[recv], 1.0).astype(np.float64)
    lam = np.ascontiguousarray(lam)
    nb = (3 if spatial else 1) * nbasis(Np)
    out = np.empty((n, nb, nb))
    dout = np.empty((n, nb, nb)) if with_derivative else None
    qu = np.empty(n, dtype=np.int32)
    if q is not None:
        lev0 = list(G.qs).index(q)
        rtol = 0.0
    tri_lev = list(G.qs).index(TRI_ORDER)
    nlev = len(GL_ORDERS)
    (lib().orc_blocks_p1 if spatial else lib().orc_blocks)(_p(verts), _p(tets, _i32p), ctypes.c_int64(n), _p(t, _i64p), _p(f, _i32p), _p(fp, _i32p),
                     _p(recv, _i64p), _p(mu), _p(lam), ctypes.c_int(Np), ctypes.c_int(nlev), _p(G.qs, _i32p),
                     _p(G.offs, _i32p), _p(G.x), _p(G.w), ctypes.c_int(lev0), ctypes.c_double(rtol),
                     ctypes.c_int(tri_lev), ctypes.c_int(regions_mask), ctypes.c_int(nthreads), _p(out),
                     _p(dout) if dout is not None else None, _p(qu, _i32p))
    return out, dout, qu, recv


def assemble(verts, tets, mu_tet, refl, Np, q=None, rtol=1e-13, with_derivative=False, topo=None,
             nthreads=0, spatial=0) -> Operator:
    """The whole operator B (all 12 face pairs of every tet), Sec. 3.2
    (spatial=1: the linear spatial basis, see blocks_for_pairs)."""
    topo = topo or topology(tets)
    nt = tets.shape[0]
    t, f, fp = pair_list(nt)
    out, dout, qu, recv = blocks_for_pairs(verts, tets, topo, mu_tet, refl, Np, t, f, fp, q=q, rtol=rtol,
                                           with_derivative=with_derivative, nthreads=nthreads, spatial=spatial)
    ns = 3 if spatial else 1
    nb = ns * nbasis(Np)
    return Operator(Np=Np, blocks=out.reshape(4 * nt, 3, nb, nb), dest=recv.reshape(4 * nt, 3),
                    dblocks=None if dout is None else dout.reshape(4 * nt, 3, nb, nb), q_used=qu, ns=ns)


def transmission(cos_r, c_ratio, z_src, z_dst) -> float:
    """Acoustic transmission probability across an interface (Sec. 3.3):
    lambda_t = 4 z_i z_j cos(theta_r) cos(theta_t) / (z_i cos(theta_r) + z_j cos(theta_t))^2
    with sin(theta_t) = (c_i / c_j) sin(theta_r) (Snell's law), zero beyond the
    critical angle; j is the tet the ray leaves (z_src), i the one it enters."""
    return float(lib().orc_transmission(cos_r, c_ratio, z_src, z_dst))


def assemble_media(verts, tets, mu_tet, c_tet, rhof_tet, refl, Np, q=None, rtol=1e-13, topo=None,
                   nthreads=0, with_derivative=False) -> Operator:
    """B for heterogeneous media (Sec. 3.2 Eq. B4DInt with the transmission
    law of Sec. 3.3): per-tet propagation speed c and fluid density rho_f
    (impedance z = rho_f c).  A ray leaving tet j through an interior face
    enters the neighbour i with probability lambda_t(theta_r), its tangential
    direction scaled by c_i / c_j (the receiving Zernike argument is the
    transmitted direction rescaled to the unit disc), and returns into tet j
    by specular reflection with probability 1 - lambda_t (rblocks, received by
    the exit face's own row).  Boundary faces reflect with weight r as in
    assemble.  With equal media everywhere this is assemble's operator and the
    rblocks vanish.  with_derivative adds d(blocks)/d(mu_t) (dblocks) and
    d(rblocks)/d(mu_t) (drblocks): both parts cross tet t, whose damping they carry."""
    G = gl_table()
    topo = topo or topology(tets)
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    nt = tets.shape[0]
    t, f, fp = pair_list(nt)
    recv = np.ascontiguousarray(topo.recv[4 * t + fp], dtype=np.int64)
    bnd = topo.boundary[recv]
    c_tet = np.broadcast_to(np.asarray(c_tet, dtype=np.float64), (nt,))
    z_tet = c_tet * np.broadcast_to(np.asarray(rhof_tet, dtype=np.float64), (nt,))
    i = recv // 4
    mu = np.ascontiguousarray(np.asarray(mu_tet, dtype=np.float64)[t])
    refl_row = np.broadcast_to(np.asarray(refl, dtype=np.float64), (4 * nt,))
    nb = nbasis(Np)
    if q is not None:
        lev0, rtol = list(G.qs).index(q), 0.0
    else:
        lev0 = 1
    tri_lev = list(G.qs).index(TRI_ORDER)

    def run(sel, rows, kind, lam):
        n = int(np.count_nonzero(sel))
        out = np.zeros((n, nb, nb))
        dout = np.zeros((n, nb, nb)) if with_derivative else None
        qu = np.empty(n, dtype=np.int32)
        if n == 0:
            return out, dout, qu
        a = lambda v, dt=np.float64: np.ascontiguousarray(np.asarray(v)[sel], dtype=dt)  # noqa: E731
        lib().orc_blocks_media(_p(verts), _p(tets, _i32p), ctypes.c_int64(n), _p(a(t, np.int64), _i64p),
                               _p(a(f, np.int32), _i32p), _p(a(fp, np.int32), _i32p), _p(a(rows, np.int64), _i64p),
                               _p(a(mu)), _p(a(lam)), _p(a(kind, np.int32), _i32p), _p(a(c_tet[i] / c_tet[t])),
                               _p(a(z_tet[t])), _p(a(z_tet[i])), ctypes.c_int(Np), ctypes.c_int(len(GL_ORDERS)),
                               _p(G.qs, _i32p), _p(G.offs, _i32p), _p(G.x), _p(G.w), ctypes.c_int(lev0),
                               ctypes.c_double(rtol), ctypes.c_int(tri_lev), ctypes.c_int(0x0F),
                               ctypes.c_int(nthreads), _p(out), _p(dout) if dout is not None else None,
                               _p(qu, _i32p))
        return out, dout, qu

    everything = np.ones(t.size, dtype=bool)
    lam = np.where(bnd, refl_row[recv], 1.0)
    kind = np.where(bnd, 0, 1)
    b1, d1, q1 = run(everything, recv, kind, lam)
    rb = np.zeros((t.size, nb, nb))
    b2, d2, _ = run(~bnd, 4 * t + fp, np.full(t.size, 2), np.ones(t.size))
    rb[~bnd] = b2
    shape = (4 * nt, 3, nb, nb)
    op = Operator(Np=Np, blocks=b1.reshape(shape), dest=recv.reshape(4 * nt, 3), q_used=q1,
                  rblocks=rb.reshape(shape), rdest=(4 * t + fp).reshape(4 * nt, 3))
    if with_derivative:
        drb = np.zeros((t.size, nb, nb))
        drb[~bnd] = d2
        op.dblocks = d1.reshape(shape)
        op.drblocks = drb.reshape(shape)
    return op


def mc_block_media(verts, tets, t, f, fp, recv_row, mu, kind, c_ratio, z_src, z_dst, Np, nsamp=10 ** 7, seed=1,
                   nthreads=0):
    """Monte Carlo ray tracing of one block across an interface (kind 1: the
    transmitted part, received by recv_row; kind 2: the reflected part, received
    by row 4t + fp): (mean, standard error)."""
    nb = nbasis(Np)
    mean = np.empty((nb, nb))
    se = np.empty((nb, nb))
    lib().orc_mc_block_media(_p(np.ascontiguousarray(verts, dtype=np.float64)),
                             _p(np.ascontiguousarray(tets, dtype=np.int32), _i32p), ctypes.c_int64(t),
                             ctypes.c_int(f), ctypes.c_int(fp), ctypes.c_int64(recv_row), ctypes.c_double(mu),
                             ctypes.c_int(kind), ctypes.c_double(c_ratio), ctypes.c_double(z_src),
                             ctypes.c_double(z_dst), ctypes.c_int(Np), ctypes.c_int64(nsamp), ctypes.c_uint64(seed),
                             ctypes.c_int(nthreads), _p(mean), _p(se))
    return mean, se


def region_cos_measure(verts, tets, t, f, fp, region, q=32):
    """Int cos(theta) dw over one of the seven direction regions by quadrature."""
    x, w = np.polynomial.legendre.leggauss(q)
    return lib().orc_region_cos_measure(_p(np.ascontiguousarray(verts, dtype=np.float64)),
                                        _p(np.ascontiguousarray(tets, dtype=np.int32), _i32p), ctypes.c_int64(t),
                                        ctypes.c_int(f), ctypes.c_int(fp), ctypes.c_int(region), ctypes.c_int(q),
                                        _p(x), _p(w))


def spatial(verts, tets, t, f, direction, mu, nq=TRI_ORDER):
    """S_{f->fp}(d), dS/dmu and the clipped area for the three fp != f (ascending)."""
    x, w = np.polynomial.legendre.leggauss(nq)
    S = np.empty(3)
    dS = np.empty(3)
    A = np.empty(3)
    d = np.ascontiguousarray(direction, dtype=np.float64)
    lib().orc_spatial(_p(np.ascontiguousarray(verts, dtype=np.float64)),
                      _p(np.ascontiguousarray(tets, dtype=np.int32), _i32p), ctypes.c_int64(t), ctypes.c_int(f),
                      _p(d), ctypes.c_double(mu), ctypes.c_int(nq), _p(x), _p(w), _p(S), _p(dS), _p(A))
    return S, dS, A


def spatial_p1(verts, tets, t, f, fp, recv_row, direction, mu, nq=TRI_ORDER):
    """The linear-basis spatial matrix S[b][a] = Int (sqrt|T_l| phi_a)(s)
    (sqrt|T_l'| psi_b)(exit point) exp(-mu L(s)) ds over the source points of
    face (t, f) whose ray in `direction` leaves through face fp (received by
    recv_row), by clipping; and its mu-derivative.  [3, 3] each."""
    x, w = np.polynomial.legendre.leggauss(nq)
    S = np.empty(9)
    dS = np.empty(9)
    lib().orc_spatial_p1(_p(np.ascontiguousarray(verts, dtype=np.float64)),
                         _p(np.ascontiguousarray(tets, dtype=np.int32), _i32p), ctypes.c_int64(t), ctypes.c_int(f),
                         ctypes.c_int(fp), ctypes.c_int64(recv_row),
                         _p(np.ascontiguousarray(direction, dtype=np.float64)), ctypes.c_double(mu), ctypes.c_int(nq),
                         _p(x), _p(w), _p(S), _p(dS))
    return S.reshape(3, 3), dS.reshape(3, 3)


def mc_block(verts, tets, t, f, fp, recv_row, mu, lam, Np, nsamp=10 ** 7, seed=1, nthreads=0, spatial=0):
    """Brute-force Monte Carlo ray tracing of one block: (mean, standard error)
    (spatial=1: the linear spatial basis, the score weighted by the source
    function at the ray's start and the receiving function at its exit)."""
    nb = (3 if spatial else 1) * nbasis(Np)
    mean = np.empty((nb, nb))
    se = np.empty((nb, nb))
    (lib().orc_mc_block_p1 if spatial else lib().orc_mc_block)(_p(np.ascontiguousarray(verts, dtype=np.float64)),
                       _p(np.ascontiguousarray(tets, dtype=np.int32), _i32p), ctypes.c_int64(t), ctypes.c_int(f),
                       ctypes.c_int(fp), ctypes.c_int64(recv_row), ctypes.c_double(mu), ctypes.c_double(lam),
                       ctypes.c_int(Np), ctypes.c_int64(nsamp), ctypes.c_uint64(seed), ctypes.c_int(nthreads),
                       _p(mean), _p(se))
    return mean, se


# ---------------------------------------------------------------------------
# Operator application and solves (Sec. 2, Eqs. NSum and GovIE)
# ---------------------------------------------------------------------------

def apply(op: Operator, x: np.ndarray, trans: bool = False, x0=None, alpha=1.0, nthreads=0) -> np.ndarray:
    """y = x0 + alpha * B x (or B^T x), x of shape [nrows, nb] (one right-hand side)."""
    nb = op.nb
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(op.nrows, nb)
    y = np.empty_like(x)
    blocks = np.ascontiguousarray(op.blocks)
    dest = np.ascontiguousarray(op.dest, dtype=np.int64)
    x0p = None if x0 is None else _p(np.ascontiguousarray(x0, dtype=np.float64).reshape(op.nrows, nb))
    lib().orc_apply(ctypes.c_int64(op.nrows), ctypes.c_int(nb), _p(blocks), _p(dest, _i64p), _p(x), x0p,
                    ctypes.c_double(alpha), ctypes.c_int(1 if trans else 0), ctypes.c_int(nthreads), _p(y))
    if op.rblocks is not None:
        rb = np.ascontiguousarray(op.rblocks)
        rd = np.ascontiguousarray(op.rdest, dtype=np.int64)
        y2 = np.empty_like(x)
        lib().orc_apply(ctypes.c_int64(op.nrows), ctypes.c_int(nb), _p(rb), _p(rd, _i64p), _p(x), _p(y),
                        ctypes.c_double(alpha), ctypes.c_int(1 if trans else 0), ctypes.c_int(nthreads), _p(y2))
        y = y2
    return y


def dense(op: Operator) -> np.ndarray:
    """B as a dense [nrows*nb, nrows*nb] matrix (small meshes only)."""
    nb = op.nb
    n = op.nrows * nb
    M = np.zeros((n, n))
    for J in range(op.nrows):
        for k in range(3):
            R = int(op.dest[J, k])
            M[R * nb:(R + 1) * nb, J * nb:(J + 1) * nb] += op.blocks[J, k]
            if op.rblocks is not None:
                R = int(op.rdest[J, k])
                M[R * nb:(R + 1) * nb, J * nb:(J + 1) * nb] += op.rblocks[J, k]
    return M


def p1_coeffs() -> np.ndarray:
    """C[a][k] of the linear spatial basis: sqrt|T| phi_a = sum_k C[a][k] l_k
    with l_k the barycentric coordinate of the face's k-th vertex (frame order)."""
    out = np.empty(9)
    lib().orc_p1_coeffs(_p(out))
    return out.reshape(3, 3)


def source_vector(verts, tets, rows, Np, weights=None, spatial=0) -> np.ndarray:
    """Galerkin coefficients of a unit isotropic density on boundary face rows:
    rho0 = 1 on Q_row projects onto b_l Z_0^0 with coefficient sqrt(|T_l|) * 1
    (b_l = 1/sqrt|T_l|, the Zernike (0,0) inverse norm 1/pi times the disc area pi),
    and to zero on every other basis function (Sec. 3.1-3.2).  [nrows, nb]
    (spatial=1: nb = 3 nbasis(Np); the linear functions have zero mean, so the
    coefficient sits on the constant one, index 0, as well)."""
    nb = (3 if spatial else 1) * nbasis(Np)
    area = face_areas(verts, tets)
    x = np.zeros((4 * tets.shape[0], nb))
    w = np.ones(len(rows)) if weights is None else weights
    for r, wt in zip(np.atleast_1d(rows), np.atleast_1d(w)):
        x[int(r), 0] += wt * np.sqrt(area[int(r)])
    return x


def face_frames(verts, tets):
    """Frame of every row 4t + f (the convention of dfm_oracle.c, Sec. 3.3 leaves
    it open): origin at the first face vertex v_{f+1}, e1 = unit(v_{f+2} - v_{f+1}),
    n = unit normal towards v_f, e2 = n x e1.  Returns (e1, e2, n) [rows, 3] each."""
    nt = tets.shape[0]
    e1 = np.empty((4 * nt, 3))
    e2 = np.empty((4 * nt, 3))
    nn = np.empty((4 * nt, 3))
    for f in range(4):
        p0, p1, p2 = (verts[tets[:, (f + 1 + k) % 4]] for k in range(3))
        apex = verts[tets[:, f]]
        a = p1 - p0
        c = np.cross(a, p2 - p0)
        c *= np.sign(np.einsum("ij,ij->i", c, apex - p0))[:, None]
        n = c / np.linalg.norm(c, axis=1)[:, None]
        u = a / np.linalg.norm(a, axis=1)[:, None]
        e1[f::4], nn[f::4], e2[f::4] = u, n, np.cross(n, u)
    return e1, e2, nn


def source_directed(verts, tets, rows, Np, dirs=None, combine=False, spatial=0) -> np.ndarray:
    """Galerkin coefficients of a unit density travelling in one direction d on
    each listed face (Sec. 4.1, Eq. RhoNeumann for d = the inward normal).  The
    density delta(p - p_d), p_d = (d.e1, d.e2), projected onto the basis of
    Eq. FBApprox: coefficient (n, m) = (inverse norm N_nm) * <delta, Z_n^m> *
    <1_T, 1/sqrt|T|> = N_nm Z_n^m(p_d) sqrt|T|.  dirs None = inward normals.
    Returns [n_src, rows, nb], or [rows, nb] summed when combine is set
    (spatial=1: nb = 3 nbasis(Np), a constant density projects onto the
    constant spatial function only, the first nbasis(Np) entries)."""
    nz = nbasis(Np)
    nb = (3 if spatial else 1) * nz
    rows = np.atleast_1d(np.asarray(rows, dtype=np.int64))
    area = face_areas(verts, tets)
    e1, e2, nn = face_frames(verts, tets)
    inv = zernike_invnorm(Np)
    out = np.zeros((rows.size, 4 * tets.shape[0], nb))
    for s, r in enumerate(rows):
        if dirs is None:
            p = (0.0, 0.0)
        else:
            d = np.asarray(dirs[s], dtype=np.float64)
            d = d / np.linalg.norm(d)
            if not d @ nn[r] > 0:
                raise ValueError("direction does not enter the tet")
            p = (d @ e1[r], d @ e2[r])
        out[s, r, :nz] = inv * zernike(Np, p[0], p[1])[0] * np.sqrt(area[r])
    return out.sum(axis=0) if combine else out


def point_source(verts, tets, r0, Np, mu_tet, refl, strength=1.0, nq=48, topo=None) -> np.ndarray:
    """Galerkin coefficients of a point source at r0 (Sec. 4.2, Eq. SourceRho)
    in uniform media.  Rays leave r0 in every direction, cross the tet that
    holds them and enter the next tet through a face F that does not contain
    r0; on F the density is strength * cos(theta) exp(-mu R) / R^2 times a
    delta at the ray's inward direction u = unit(s - r0), R = |s - r0|, theta
    the angle between u and the receiving face's inward normal (Eq. SourceRho
    with strength = rho_f omega^2 / (16 pi^2 c); the paper writes the
    direction from the source's side, r0 - s, in that tet's own frame).  It
    is received by the row across F (the neighbour's face), or by F's own row
    with weight r and the specularly reflected direction (same tangential
    components) on the boundary.  Projection onto the basis of Eq. FBApprox:
        a[row][(n,m)] = N_nm / sqrt|F| Int_F strength cos exp(-mu R)/R^2 Z_n^m(p(u)) ds
    by collapsed tensor Gauss-Legendre of order nq.  r0 inside a tet uses its
    four faces; r0 on a face, an edge or at a vertex uses, in every tet whose
    closure holds it, the faces that do not contain it.  [nrows, nb]."""
    topo = topo or topology(tets)
    nt = tets.shape[0]
    nb = nbasis(Np)
    inv = zernike_invnorm(Np)
    e1, e2, nn = face_frames(verts, tets)
    area = face_areas(verts, tets)
    refl_row = np.broadcast_to(np.asarray(refl, dtype=np.float64), (4 * nt,))
    mu_tet = np.broadcast_to(np.asarray(mu_tet, dtype=np.float64), (nt,))
    r0 = np.asarray(r0, dtype=np.float64)
    gx, gw = np.polynomial.legendre.leggauss(nq)
    u = 0.5 * (1 + gx)[:, None] * np.ones(nq)[None, :]
    v = (1 - u) * 0.5 * (1 + gx)[None, :]
    wq = (gw[:, None] * gw[None, :]) * 0.25 * (1 - u)  # x 2|F| below
    out = np.zeros((4 * nt, nb))
    for k in range(nt):
        P = verts[tets[k]]
        lam = np.linalg.solve(np.vstack([P.T, np.ones(4)]), np.append(r0, 1.0))  # barycentric coordinates
        if lam.min() < -1e-12:
            continue
        for l in range(4):
            if lam[l] <= 1e-12:  # r0 lies on face l (opposite vertex l)
                continue
            row = 4 * k + l
            rec = int(topo.recv[row])
            wgt = refl_row[row] if topo.boundary[row] else 1.0
            p0, p1, p2 = (verts[tets[k, (l + 1 + i) % 4]] for i in range(3))
            s = p0 + u[..., None] * (p1 - p0) + v[..., None] * (p2 - p0)
            d = s - r0
            R = np.linalg.norm(d, axis=-1)
            uv = d / R[..., None]
            cos = uv @ (-nn[row])  # the ray leaves tet k through F: outward normal of (k, l)
            ker = (wq * 2 * area[row] * cos * np.exp(-mu_tet[k] * R) / R ** 2).reshape(-1)
            Z = zernike(Np, (uv @ e1[rec]).reshape(-1), (uv @ e2[rec]).reshape(-1))
            out[rec] += wgt * strength * inv * (ker @ Z) / np.sqrt(area[row])
    return out


def tet_density(verts, tets, mu_tet, Np, rho, nq=48, rtol=1e-11, nthreads=0, spatial=0) -> np.ndarray:
    """rho_T at every tet centroid (Sec. 4.1, Eq. IntDens) for rho [rows, nb]:
    the per-tet functional g_t of interior_g applied to the tet's four rows
    (nq=None: adaptive cubature to rtol, all tets in parallel; spatial=1: the
    linear spatial basis, one tet after the other)."""
    if spatial:
        cen = centroids(verts, tets)
        mu_b = np.broadcast_to(np.asarray(mu_tet, dtype=np.float64), (tets.shape[0],))
        out = np.empty(tets.shape[0])
        for t in range(tets.shape[0]):
            g, _ = interior_g(verts, tets, t, cen[t], float(mu_b[t]), Np, nq=nq, rtol=rtol, spatial=1)
            out[t] = np.sum(g * rho[4 * t:4 * t + 4])
        return out
    if nq is None:
        nt = tets.shape[0]
        nb = nbasis(Np)
        x, w = np.polynomial.legendre.leggauss(8)
        g = np.empty((nt, 4, nb))
        dg = np.empty((nt, 4, nb))
        lib().orc_centroid_g_adaptive(_p(np.ascontiguousarray(verts, dtype=np.float64)),
                                      _p(np.ascontiguousarray(tets, dtype=np.int32), _i32p), ctypes.c_int64(nt),
                                      _p(np.ascontiguousarray(np.broadcast_to(np.asarray(mu_tet, dtype=np.float64),
                                                                              (nt,)))),
                                      ctypes.c_int(Np), ctypes.c_double(rtol), ctypes.c_int(8), _p(x), _p(w),
                                      ctypes.c_int(nthreads), _p(g), _p(dg))
        return np.einsum("tlk,tlk->t", g, rho.reshape(nt, 4, nb))
    cen = centroids(verts, tets)
    out = np.empty(tets.shape[0])
    for t in range(tets.shape[0]):
        g, _ = interior_g(verts, tets, t, cen[t], float(mu_tet[t]), Np, nq=nq)
        out[t] = np.sum(g * rho[4 * t:4 * t + 4])
    return out


def solve_dense(op: Operator, rho0: np.ndarray) -> np.ndarray:
    """rho = (I - B)^{-1} rho0 by LU (Eq. GovIE); small meshes."""
    M = np.eye(op.nrows * op.nb) - dense(op)
    return np.linalg.solve(M, rho0.reshape(-1)).reshape(op.nrows, op.nb)


def neumann(op: Operator, rho0: np.ndarray, tol=1e-10, maxit=100000):
    """Neumann series rho = sum_n B^n rho0 (Eq. NSum), iterated as x <- rho0 + B x
    until ||x_{k+1} - x_k|| <= tol ||x_{k+1}||."""
    x = rho0.copy()
    for it in range(1, maxit + 1):
        xn = apply(op, x, x0=rho0)
        if np.linalg.norm(xn - x) <= tol * np.linalg.norm(xn):
            return xn, it
        x = xn
    return x, -maxit


def gmres(matvec, b: np.ndarray, tol=1e-12, restart=200, maxit=20000, x0=None):
    """Restarted GMRES (modified Gram-Schmidt Arnoldi, Givens rotations) on a
    flat vector; stops on the true residual ||b - A x|| <= tol ||b||."""
    b = b.reshape(-1)
    x = np.zeros_like(b) if x0 is None else x0.reshape(-1).copy()
    bn = np.linalg.norm(b)
    if bn == 0:
        return x, 0
    total = 0
    while total < maxit:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bn:
            return x, total
        m = restart
        V = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(m):
            w = matvec(V[k])
            for i in range(k + 1):
                H[i, k] = np.dot(V[i], w)
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                a, c = H[i, k], H[i + 1, k]
                H[i, k] = cs[i] * a + sn[i] * c
                H[i + 1, k] = -sn[i] * a + cs[i] * c
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / den
            sn[k] = H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            total += 1
            k_done = k + 1
            if abs(g[k + 1]) <= 0.5 * tol * bn or total >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        x = x + V[:k_done].T @ y
    r = b - matvec(x)
    return x, (total if np.linalg.norm(r) <= tol * bn else -total)


def solve_gmres(op: Operator, rho0: np.ndarray, tol=1e-12, restart=200, maxit=20000, trans=False, nthreads=0):
    """(I - B) x = rho0 (or (I - B)^T x = rho0) by restarted GMRES, FP64."""
    nb = op.nb

    def mv(v):
        return apply(op, v.reshape(op.nrows, nb), trans=trans, x0=v.reshape(op.nrows, nb), alpha=-1.0,
                     nthreads=nthreads).reshape(-1)

    x, it = gmres(mv, rho0.reshape(-1), tol=tol, restart=restart, maxit=maxit)
    return x.reshape(op.nrows, nb), it


def residual(op: Operator, x: np.ndarray, rho0: np.ndarray) -> float:
    """||rho0 - (I - B) x|| / ||rho0|| in FP64."""
    r = rho0 - apply(op, x, x0=x, alpha=-1.0)
    return float(np.linalg.norm(r) / np.linalg.norm(rho0))


# ---------------------------------------------------------------------------
# Interior density and the adjoint gradient (Sec. 4.1, Eq. IntDens)
# ---------------------------------------------------------------------------

def centroids(verts, tets):
    return verts[tets].mean(axis=1)


def interior_g(verts, tets, t, r, mu, Np, nq=48, rtol=1e-11, spatial=0):
    """g[4, nb] and dg/dmu with rho_T(r) = sum_{l,nm} rho_(t,l,nm) g[l,nm]
    (Sec. 4.1, Eq. IntDens): a fixed collapsed Gauss rule of order nq on each
    face, or, with nq=None, adaptive 4-way refinement of each face to rtol.
    spatial=1: the linear spatial basis, g[4, 3 nb] with the integrand weighted
    by each face function sqrt|T_l| phi_s at the face point."""
    nb = (3 if spatial else 1) * nbasis(Np)
    g = np.empty((4, nb))
    dg = np.empty((4, nb))
    rr = np.ascontiguousarray(r, dtype=np.float64)
    if nq is None:
        x, w = np.polynomial.legendre.leggauss(8)
        (lib().orc_interior_g_adaptive_p1 if spatial else lib().orc_interior_g_adaptive)(
                                      _p(np.ascontiguousarray(verts, dtype=np.float64)),
                                      _p(np.ascontiguousarray(tets, dtype=np.int32), _i32p), ctypes.c_int64(int(t)),
                                      _p(rr), ctypes.c_double(mu), ctypes.c_int(Np), ctypes.c_double(rtol),
                                      ctypes.c_int(8), _p(x), _p(w), _p(g), _p(dg))
        return g, dg
    x, w = np.polynomial.legendre.leggauss(nq)
    (lib().orc_interior_g_p1 if spatial else lib().orc_interior_g)(_p(np.ascontiguousarray(verts, dtype=np.float64)),
                         _p(np.ascontiguousarray(tets, dtype=np.int32), _i32p), ctypes.c_int64(int(t)), _p(rr),
                         ctypes.c_double(mu), ctypes.c_int(Np), ctypes.c_int(nq), _p(x), _p(w), _p(g), _p(dg))
    return g, dg


def interior_g_split(verts, tets, t, r, mu, Np, n=16):
    """The functional of interior_g by a rule that stays exact when r is close
    to a face or the foot F of r (height h) is close to a face edge: each face
    is split at F into three signed triangles (F, A, B) over its edges and
    integrated in polar coordinates seen from r.  The area element times
    cos / R^2 is sin(phi) dphi dpsi (psi the azimuth about the face normal,
    phi the polar angle up to the edge, phi in [0, atan(l / h)], l = |X - F|
    for the edge point X at that azimuth).  The azimuth is sampled through the
    edge point X = M + u t (M the foot of the perpendicular from F to the
    line AB, t its unit direction, d = |M - F|): dpsi = d du / (d^2 + u^2),
    u = c tan(s) with c = sqrt(h^2 + d^2) and Gauss nodes uniform in s, the
    edge cut at M (or at its middle in s when M lies outside the edge).  The
    integrand, with exp(-mu h / cos(phi)) and the Zernike vector of the
    direction, varies in u on the scale c, so n-point Gauss-Legendre in s and
    in phi converges fast whether r is close to the face (h << d) or F close
    to an edge's line (d << h).  Returns g[4, nb] (no dg)."""
    nb = nbasis(Np)
    e1, e2, nn = face_frames(verts, tets)
    area = face_areas(verts, tets)
    x, w = np.polynomial.legendre.leggauss(n)
    x01, w01 = 0.5 * (x + 1), 0.5 * w
    r = np.asarray(r, dtype=np.float64)
    g = np.zeros((4, nb))
    for l in range(4):
        row = 4 * t + l
        P = verts[[tets[t, (l + 1 + k) % 4] for k in range(3)]]
        n_in, a1, a2 = nn[row], e1[row], e2[row]
        h = float((r - P[0]) @ n_in)  # r lies on the inner side
        F = r - h * n_in
        orient = np.sign(np.cross(P[1] - P[0], P[2] - P[0]) @ n_in)
        p2 = [np.array([(X - F) @ a1, (X - F) @ a2]) for X in P]  # vertices in the face plane, F at 0
        acc = np.zeros(nb)
        for k in range(3):
            A, B = p2[k], p2[(k + 1) % 3]
            tdir = (B - A) / np.linalg.norm(B - A)
            d = abs(A[0] * tdir[1] - A[1] * tdir[0])  # distance from F to the line AB
            if d < 1e-15 * np.linalg.norm(B - A):
                continue
            sign = np.sign(A[0] * B[1] - A[1] * B[0])  # orientation of the triangle (F, A, B)
            uA, uB = A @ tdir, B @ tdir
            M = A - uA * tdir
            c = np.hypot(h, d)
            sA, sB = np.arctan2(uA, c), np.arctan2(uB, c)
            cut = 0.0 if sA < 0.0 < sB else 0.5 * (sA + sB)
            for s0, s1 in ((sA, cut), (cut, sB)):
                sv = s0 + (s1 - s0) * x01
                u = c * np.tan(sv)
                ell = np.sqrt(d * d + u * u)
                eh = (M[None, :] + u[:, None] * tdir[None, :]) / ell[:, None]
                Phi = np.arctan2(ell, h)
                phi = Phi[:, None] * x01[None, :]
                jac = (s1 - s0) * w01 * c / np.cos(sv) ** 2 * d / ell ** 2  # dpsi per unit of s
                wt = jac[:, None] * (Phi[:, None] * w01[None, :]) * np.sin(phi) * np.exp(-mu * h / np.cos(phi))
                dx = -np.sin(phi) * eh[:, 0:1]  # tangential part of unit(r - s) in the face frame
                dy = -np.sin(phi) * eh[:, 1:2]
                Z = zernike(Np, dx.reshape(-1), dy.reshape(-1))
                acc += orient * sign * (wt.reshape(-1) @ Z)
        g[l] = acc / np.sqrt(area[row])
    return g


def receiver_functional(verts, tets, mu_tet, Np, receiver, nq=48):
    """J(rho) = mean over receiver tets e of rho_T(centroid_e) = gvec . rho.
    Returns gvec [nrows, nb] and dgvec/dmu_e stacked per receiver tet."""
    nb = nbasis(Np)
    gvec = np.zeros((4 * tets.shape[0], nb))
    dg = {}
    cen = centroids(verts, tets)
    for e in np.atleast_1d(receiver):
        g, d = interior_g(verts, tets, int(e), cen[int(e)], float(mu_tet[int(e)]), Np, nq=nq)
        gvec[4 * e:4 * e + 4] += g / len(receiver)
        dg[int(e)] = d / len(receiver)
    return gvec, dg


def gradient(op: Operator, rho: np.ndarray, lam: np.ndarray, dg: dict, nt: int) -> np.ndarray:
    """dJ/dmu_e = (dg/dmu_e) . rho + sum_{blocks of tet e} lam_R^T (dB/dmu_e) rho_J,
    with (I - B)^T lam = g (the adjoint equation).  op must carry dblocks."""
    nb = op.nb
    grad = np.zeros(nt)
    db = op.dblocks.reshape(nt, 4, 3, nb, nb)
    dest = op.dest.reshape(nt, 4, 3)
    rho_t = rho.reshape(nt, 4, nb)
    lam_r = lam[dest]  # [nt, 4, 3, nb]
    grad += np.einsum("tfka,tfkab,tfb->t", lam_r, db, rho_t)
    if op.drblocks is not None:  # heterogeneous media: the interface reflections cross tet e too
        lam_rr = lam[op.rdest.reshape(nt, 4, 3)]
        grad += np.einsum("tfka,tfkab,tfb->t", lam_rr, op.drblocks.reshape(nt, 4, 3, nb, nb), rho_t)
    for e, d in dg.items():
        grad[e] += float(np.sum(d * rho[4 * e:4 * e + 4]))
    return grad
