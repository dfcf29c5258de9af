"""Seeded synthetic inputs for discrete flow mapping on tetrahedral meshes.

This module produces *inputs only*: mesh arrays, damping fields, source rows,
receiver sets and sampled element lists.  It holds none of the method's
arithmetic (no face frames, no operator entries, no neighbour search), so
the CUDA path and the CPU oracle can both consume it without sharing code.

Meshes are jittered Kuhn cubes: the unit cube [0,1]^3 split into n^3 cells of
side h = 1/n, each cell cut into six tetrahedra (one per permutation of the
axes), interior vertices perturbed per coordinate by U[-jitter*h, +jitter*h]
from a seeded PCG64 stream.  The paper's own meshes (a 972-tet cuboid, Sec. 4.1,
and a proprietary vehicle cavity, Sec. 4.2) are not published; these meshes
stand in for them.

All random draws use numpy's PCG64 with explicit seeds:
mesh jitter seed 0, damping field seed 1, source rows seed 2, FD elements seed 3.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

# Axis permutations in a fixed order; tet 6*c + k of cell c uses _PERMS[k].
_PERMS = tuple(itertools.permutations((0, 1, 2)))


@dataclass(frozen=True)
class KuhnMesh:
    """A Kuhn-split cube mesh.

    verts: float64 [nv, 3]; tets: int32 [6 n^3, 4] (positive orientation
    before jitter); n: cells per axis; h: cell size.  Tet 6*c + k belongs to
    cell c = i + n*(j + n*k) with cell corner (i, j, k)*h.
    """

    verts: np.ndarray
    tets: np.ndarray
    n: int
    h: float

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    @property
    def n_rows(self) -> int:
        return 4 * self.n_tets


def _vid(i, j, k, n):
    return i + (n + 1) * (j + (n + 1) * k)


def kuhn_cube_mesh(n: int, jitter: float = 0.2, seed: int = 0) -> KuhnMesh:
    """Unit cube with n^3 cells, each split into 6 tets; interior vertices jittered.

    jitter is the half-width of the uniform perturbation in units of h; 0 gives
    the regular Kuhn split.  Boundary vertices are never moved, so the six cube
    faces stay planar.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    g = np.arange(n + 1, dtype=np.float64) * h
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)  # index i + (n+1)(j + (n+1)k)

    ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # cell id c = i + n*(j + n*k): order cells by k, then j, then i
    ci = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
    order = np.lexsort((ci[:, 0], ci[:, 1], ci[:, 2]))
    ci = ci[order]
    tets = np.empty((n ** 3, 6, 4), dtype=np.int64)
    unit = np.eye(3, dtype=np.int64)
    for p, perm in enumerate(_PERMS):
        c0 = ci
        c1 = c0 + unit[perm[0]]
        c2 = c1 + unit[perm[1]]
        c3 = c0 + 1
        corners = [c0, c1, c2, c3]
        ids = [_vid(c[:, 0], c[:, 1], c[:, 2], n) for c in corners]
        tets[:, p, :] = np.stack(ids, axis=1)
    tets = tets.reshape(-1, 4)
    # positive orientation on the unjittered grid (swap the last two vertices if needed)
    a, b, c, d = (verts[tets[:, k]] for k in range(4))
    vol6 = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a)
    neg = vol6 < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()

    if jitter > 0 and n > 1:
        rng = np.random.Generator(np.random.PCG64(seed))
        delta = rng.uniform(-jitter * h, jitter * h, size=verts.shape)
        idx = np.arange(verts.shape[0])
        vi = idx % (n + 1)
        vj = (idx // (n + 1)) % (n + 1)
        vk = idx // ((n + 1) ** 2)
        interior = (vi > 0) & (vi < n) & (vj > 0) & (vj < n) & (vk > 0) & (vk < n)
        verts = verts + delta * interior[:, None]
    return KuhnMesh(verts=np.ascontiguousarray(verts), tets=np.ascontiguousarray(tets.astype(np.int32)),
                    n=n, h=h)


def _grid_index(mesh: KuhnMesh, vids: np.ndarray) -> np.ndarray:
    n = mesh.n
    return np.stack([vids % (n + 1), (vids // (n + 1)) % (n + 1), vids // ((n + 1) ** 2)], axis=-1)


def boundary_faces(mesh: KuhnMesh) -> np.ndarray:
    """Rows 4*t + f whose face lies on the cube boundary, with the cube side.

    Face f of a tet is the face opposite its local vertex f.  A face is on the
    boundary when its three vertices share a grid index 0 or n on one axis.
    Returns int64 [nb, 2]: (row, side) with side = 2*axis + (0 for the low
    face, 1 for the high face); rows ascending.
    """
    n = mesh.n
    out = []
    gi = _grid_index(mesh, mesh.tets.astype(np.int64))  # [nt, 4, 3]
    for f in range(4):
        others = [k for k in range(4) if k != f]
        tri = gi[:, others, :]  # [nt, 3, 3]
        for axis in range(3):
            for hi, val in ((0, 0), (1, n)):
                on = np.all(tri[:, :, axis] == val, axis=1)
                t = np.nonzero(on)[0]
                out.append(np.stack([4 * t + f, np.full_like(t, 2 * axis + hi)], axis=1))
    res = np.concatenate(out, axis=0)
    return res[np.argsort(res[:, 0], kind="stable")]


def source_row_minus_x(mesh: KuhnMesh, point_yz=None) -> int:
    """Row of the boundary face on the x = 0 side used as a single source.

    Without point_yz: the lowest row on the x = 0 side.  With point_yz=(y, z):
    the lowest row on the x = 0 side whose triangle contains (0, y, z)
    (boundary vertices are never jittered, so containment uses grid
    coordinates exactly).
    """
    bf = boundary_faces(mesh)
    rows = bf[bf[:, 1] == 0, 0]
    if point_yz is None:
        return int(rows.min())
    y, z = point_yz
    for r in np.sort(rows):
        t, f = divmod(int(r), 4)
        vids = [int(mesh.tets[t, k]) for k in range(4) if k != f]
        p = mesh.verts[vids][:, 1:]  # (y, z) of the 3 vertices
        # barycentric containment in 2-D, tolerance for vertices/edges
        a, b, c = p
        m = np.array([[b[0] - a[0], c[0] - a[0]], [b[1] - a[1], c[1] - a[1]]])
        lam = np.linalg.solve(m, np.array([y - a[0], z - a[1]]))
        if lam[0] >= -1e-12 and lam[1] >= -1e-12 and lam.sum() <= 1 + 1e-12:
            return int(r)
    raise ValueError("point not on the x = 0 side")


@dataclass(frozen=True)
class KuhnCuboid:
    """A Kuhn-split box (0, length) x (-1/2, 1/2)^2 of cubic cells of side h = 1/n:
    nx = round(length n) cells along x, n along y and z, six tets per cell.
    verts: float64 [nv, 3], vertex (i, j, k) at index i + (nx+1)(j + (n+1)k);
    tets: int32 [6 nx n^2, 4], positively oriented before jitter."""

    verts: np.ndarray
    tets: np.ndarray
    nx: int
    n: int
    h: float
    length: float

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    @property
    def n_rows(self) -> int:
        return 4 * self.n_tets


def kuhn_cuboid_mesh(n: int, length: float = 2.0, jitter: float = 0.2, seed: int = 0) -> KuhnCuboid:
    """The cuboid cavity of the paper's verification (Sec. 4.1), (0, length) x
    (-1/2, 1/2)^2, as a Kuhn split of cubic cells with interior vertices
    jittered by U[-jitter h, jitter h] per coordinate (PCG64 seed); boundary
    vertices stay on the box so its six sides stay planar."""
    nx = int(round(length * n))
    if n < 1 or nx < 1:
        raise ValueError("need at least one cell per axis")
    h = 1.0 / n
    dims = np.array([nx, n, n])
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    g = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
    g = g[np.lexsort((g[:, 0], g[:, 1], g[:, 2]))]  # index i + (nx+1)(j + (n+1)k)
    verts = np.stack([g[:, 0] * h, g[:, 1] * h - 0.5, g[:, 2] * h - 0.5], axis=1)
    ci = np.stack(np.meshgrid(np.arange(nx), np.arange(n), np.arange(n), indexing="ij"), axis=-1).reshape(-1, 3)
    ci = ci[np.lexsort((ci[:, 0], ci[:, 1], ci[:, 2]))]

    def vid(c):
        return c[:, 0] + (nx + 1) * (c[:, 1] + (n + 1) * c[:, 2])

    tets = np.empty((ci.shape[0], 6, 4), dtype=np.int64)
    unit = np.eye(3, dtype=np.int64)
    for p, perm in enumerate(_PERMS):
        c1 = ci + unit[perm[0]]
        c2 = c1 + unit[perm[1]]
        tets[:, p, :] = np.stack([vid(ci), vid(c1), vid(c2), vid(ci + 1)], axis=1)
    tets = tets.reshape(-1, 4)
    a, b, c, d = (verts[tets[:, k]] for k in range(4))
    neg = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a) < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    if jitter > 0:
        rng = np.random.Generator(np.random.PCG64(seed))
        delta = rng.uniform(-jitter * h, jitter * h, size=verts.shape)
        interior = np.all((g > 0) & (g < dims[None, :]), axis=1)
        verts = verts + delta * interior[:, None]
    return KuhnCuboid(verts=np.ascontiguousarray(verts), tets=np.ascontiguousarray(tets.astype(np.int32)),
                      nx=nx, n=n, h=h, length=float(length))


def cuboid_rows_x0(mesh: KuhnCuboid) -> np.ndarray:
    """Rows 4t + f whose face lies on the x = 0 side of the cuboid, ascending."""
    i = mesh.tets.astype(np.int64) % (mesh.nx + 1)  # grid index along x of every tet vertex
    out = []
    for f in range(4):
        others = [k for k in range(4) if k != f]
        t = np.nonzero(np.all(i[:, others] == 0, axis=1))[0]
        out.append(4 * t + f)
    return np.sort(np.concatenate(out)).astype(np.int64)


def random_boundary_rows(mesh: KuhnMesh, count: int, seed: int = 2) -> np.ndarray:
    """count boundary rows drawn uniformly with replacement (PCG64 seed)."""
    rows = boundary_faces(mesh)[:, 0]
    rng = np.random.Generator(np.random.PCG64(seed))
    return rows[rng.integers(0, rows.shape[0], size=count)].astype(np.int64)


def uniform_mu(mesh: KuhnMesh, mu: float) -> np.ndarray:
    return np.full(mesh.n_tets, float(mu), dtype=np.float64)


def lognormal_mu(mesh: KuhnMesh, median: float = 0.05, sigma: float = 0.5, corr_cells: float = 3.0,
                 seed: int = 1) -> np.ndarray:
    """Per-tet damping mu = median * exp(sigma * G(cell)).

    G is unit-variance Gaussian white noise on the n^3 cell grid convolved with a
    Gaussian kernel of standard deviation corr_cells/sqrt(2) (truncated at 4
    standard deviations, zero padding), then divided by its theoretical standard
    deviation, which gives the correlation exp(-d^2 / (2 corr_cells^2)).  All
    six tets of a cell share G.
    """
    n = mesh.n
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n, n, n))  # axes (k, j, i)
    s = corr_cells / np.sqrt(2.0)
    rad = int(np.ceil(4 * s))
    x = np.arange(-rad, rad + 1, dtype=np.float64)
    k1 = np.exp(-0.5 * (x / s) ** 2)
    g = w
    for axis in range(3):
        g = np.apply_along_axis(lambda v: np.convolve(v, k1, mode="full")[rad:rad + n], axis, g)
    g = g / np.sqrt(np.sum(k1 ** 2) ** 3)
    gc = g.reshape(-1)  # cell id i + n*(j + n*k) since axes are (k, j, i)
    return (median * np.exp(sigma * np.repeat(gc, 6))).astype(np.float64)


def cell_tets(mesh: KuhnMesh, lo, hi) -> np.ndarray:
    """Tets of the cells with lo <= (i, j, k) < hi (per axis), ascending."""
    n = mesh.n
    lo = np.broadcast_to(np.asarray(lo), (3,))
    hi = np.broadcast_to(np.asarray(hi), (3,))
    c = np.arange(n ** 3)
    i, j, k = c % n, (c // n) % n, c // (n * n)
    sel = (i >= lo[0]) & (i < hi[0]) & (j >= lo[1]) & (j < hi[1]) & (k >= lo[2]) & (k < hi[2])
    cells = np.nonzero(sel)[0]
    return (cells[:, None] * 6 + np.arange(6)[None, :]).reshape(-1).astype(np.int64)


def fd_elements(mesh: KuhnMesh, receiver_lo, receiver_hi, count: int = 32, seed: int = 3) -> np.ndarray:
    """Elements for the finite-difference gradient check: half uniform over the
    mesh, half among the cells within 2 cells of the receiver box."""
    rng = np.random.Generator(np.random.PCG64(seed))
    half = count // 2
    far = rng.choice(mesh.n_tets, size=half, replace=False)
    lo = np.maximum(np.asarray(receiver_lo) - 2, 0)
    hi = np.minimum(np.asarray(receiver_hi) + 2, mesh.n)
    near_pool = cell_tets(mesh, lo, hi)
    near = rng.choice(near_pool, size=count - half, replace=False)
    return np.concatenate([far, near]).astype(np.int64)


# Named workloads (the five configurations the method is measured on).
def workload(name: str) -> dict:
    """Inputs of a named workload as a dict of plain numbers and arrays."""
    if name == "kuhn1_np2":  # unit cube, 6 Kuhn tets, degree <= 2
        m = kuhn_cube_mesh(1, jitter=0.0)
        return dict(name=name, mesh=m, Np=2, mu=uniform_mu(m, 0.1), refl=0.9,
                    sources=np.array([source_row_minus_x(m)]), solver="neumann", tol=1e-10)
    if name == "kuhn20_np4":  # 48,000 jittered tets, degree <= 4
        m = kuhn_cube_mesh(20, jitter=0.2, seed=0)
        return dict(name=name, mesh=m, Np=4, mu=uniform_mu(m, 0.05), refl=0.95,
                    sources=np.array([source_row_minus_x(m, (0.5, 0.5))]), solver="gmres", tol=1e-8)
    if name == "kuhn30_np4_rhs128":
        m = kuhn_cube_mesh(30, jitter=0.2, seed=0)
        rng = np.random.Generator(np.random.PCG64(2))
        mu_rhs = rng.uniform(0.01, 0.2, size=128)
        return dict(name=name, mesh=m, Np=4, mu_rhs=mu_rhs, refl=0.95,
                    sources=random_boundary_rows(m, 128, seed=2), solver="batched", tol=1e-6)
    if name == "kuhn40_np3_adjoint":
        m = kuhn_cube_mesh(40, jitter=0.2, seed=0)
        return dict(name=name, mesh=m, Np=3, mu=lognormal_mu(m), refl=0.95,
                    sources=np.array([source_row_minus_x(m, (0.5, 0.5))]),
                    receiver=cell_tets(m, 18, 22), fd=fd_elements(m, 18, 22), solver="ir", tol=1e-6)
    if name == "kuhn16_np8":  # a smaller case of the 45-function workload (98,304 rows), for profiling
        m = kuhn_cube_mesh(16, jitter=0.2, seed=0)
        return dict(name=name, mesh=m, Np=8, mu=uniform_mu(m, 0.05), refl=0.95,
                    sources=random_boundary_rows(m, 16, seed=2), receiver=cell_tets(m, 6, 10), solver="ir", tol=1e-6)
    if name == "kuhn32_np8_rhs64":
        m = kuhn_cube_mesh(32, jitter=0.2, seed=0)
        return dict(name=name, mesh=m, Np=8, mu=uniform_mu(m, 0.05), refl=0.95,
                    sources=random_boundary_rows(m, 64, seed=2), receiver=cell_tets(m, 14, 18),
                    solver="ir", tol=1e-6)
    raise KeyError(name)
